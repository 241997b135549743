"""CPU-only checks of the C ABI: the library builds, loads, and exports every
entry point include/tera.h declares; the Python binding refuses to run
without a GPU (there is no CPU path).  No compute call is made here."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "tera.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tera_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_24063_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name


def test_bounds_checking_library_exports_every_declared_symbol():
    from paper_2509_24063_gb300 import build
    lib = ctypes.CDLL(build.build(debug_bounds=True))
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2509_24063_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_version_string(libpath):
    lib = ctypes.CDLL(libpath)
    lib.tera_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tera_version()


def test_invalid_grids_rejected_on_host(libpath):
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    for lo, hi, n, w in [((0,) * 3, (10,) * 3, (2, 2, 2), 5.0),      # w == side
                         ((0,) * 3, (10,) * 3, (0, 2, 2), 1.0),      # empty axis
                         ((0,) * 3, (10,) * 3, (257, 1, 1), 0.01),   # too many boxes
                         ((5, 0, 0), (5, 10, 10), (1, 1, 1), 1.0),   # lo == hi
                         ((0,) * 3, (10,) * 3, (2, 2, 2), -1.0)]:
        g = _lib.Grid()
        for a in range(3):
            g.lo[a], g.hi[a], g.n[a] = lo[a], hi[a], n[a]
        g.w = w
        h = ctypes.c_void_p()
        assert lib.tera_ctx_create(ctypes.byref(h), ctypes.byref(g), 0, 1) == _lib.EINVAL


def test_no_cpu_fallback():
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2509_24063_gb300 as tera
    with pytest.raises(RuntimeError):
        tera.Context((0, 0, 0), (10, 10, 10), (2, 2, 2), 1.0)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2509_24063_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "tera_oracle" not in text, f


@pytest.mark.parametrize("K", [1, 2, 3, 5])
def test_reference_schedule_follows_the_interval(libpath, K):
    """tera_ref_schedule against a direct simulation of the two buffers: the
    message of iteration 0 and of every multiple of K becomes the reference;
    an iteration writes into the buffer that does not hold its reference, and
    a reference iteration's buffer is kept until the next one replaces it."""
    from paper_2509_24063_gb300.api import ref_schedule
    holder = {}   # buffer -> iteration whose message it holds
    latest = None  # latest reference iteration so far
    for t in range(0, 4 * K + 3):
        out, refb, ri = ref_schedule(t, K)
        if t == 0:
            assert refb == -1
        else:
            assert ri == latest and holder[refb] == latest
            assert out != refb  # the reference is never overwritten while read
        holder[out] = t
        if t % K == 0:
            latest = t


def test_reference_schedule_rejects_zero_interval(libpath):
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    ob, rb, ri = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    assert lib.tera_ref_schedule(3, 0, ctypes.byref(ob), ctypes.byref(rb),
                                 ctypes.byref(ri)) == _lib.EINVAL


def _key(x: float) -> int:
    """Order-preserving key of a binary64 value (-0.0 taken as +0.0)."""
    import struct
    b = struct.unpack("<Q", struct.pack("<d", x + 0.0 if x == 0.0 else x))[0]
    return b ^ 0x8000000000000000 if b < 0x8000000000000000 else b ^ 0xFFFFFFFFFFFFFFFF


def _value(k: int) -> float:
    import struct
    b = k ^ 0x8000000000000000 if k >= 0x8000000000000000 else k ^ 0xFFFFFFFFFFFFFFFF
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.mark.parametrize("lo,hi,w", [
    (0.0, 600.0, 30.0),          # exact multiples
    (-37.5, 41.3, 0.7),          # negative lo, a width with no exact binary64 value
    (12.25, 13.0, 0.1),
    (1.0e6, 1.0e6 + 3.0, 0.01),  # large coordinates: the cell edges fall between ulps
    (-0.0, 5.0, 7.0),            # a single cell
    (-1.0e-3, 1.0e-3, 1.0e-5),   # across zero
])
def test_cell_thresholds_match_the_binary64_rule(libpath, lo, hi, w):
    """tera_cell_thresholds against the rule itself, evaluated with Python's
    IEEE binary64 arithmetic: T[k] is the first value of cell k (the value
    before it lies in a lower cell), and the lookup by keys gives
    floor((x - lo) / w) for values spread over the axis and for every value
    within two ulps of each boundary."""
    import math
    import numpy as np
    from paper_2509_24063_gb300.api import cell_thresholds
    cell = lambda x: math.floor((x - lo) / w)  # noqa: E731
    n = math.floor((hi - lo) / w) + 1
    T = cell_thresholds(lo, hi, w)
    assert T.shape == (n + 1,)
    assert int(T[0]) == _key(lo) and int(T[n]) == _key(hi)
    assert np.all(T[1:] >= T[:-1])
    for k in range(1, n):
        x = _value(int(T[k]))
        assert cell(x) >= k
        assert cell(math.nextafter(x, -math.inf)) < k
    rng = np.random.default_rng(4)
    xs = list(rng.uniform(lo, hi, 2000)) + [lo, math.nextafter(hi, -math.inf)]
    for k in range(1, n):
        x = _value(int(T[k]))
        for _ in range(2):
            x = math.nextafter(x, -math.inf)
        for _ in range(5):
            xs.append(x)
            x = math.nextafter(x, math.inf)
    for x in xs:
        if not (lo <= x < hi):
            continue
        i = int(np.searchsorted(T[:n], np.uint64(_key(x)), side="right")) - 1
        assert i == cell(x), x


def test_cell_thresholds_reject_bad_arguments(libpath):
    import numpy as np
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    T = np.zeros(64, dtype=np.uint64)
    p = T.ctypes.data_as(ctypes.c_void_p)
    assert lib.tera_cell_thresholds(0.0, 10.0, 1.0, 11, p) == _lib.OK
    for args in ((0.0, 10.0, 1.0, 10), (0.0, 10.0, 1.0, 12), (0.0, 10.0, 0.0, 1),
                 (0.0, 10.0, -1.0, 11), (10.0, 0.0, 1.0, 1), (float("nan"), 10.0, 1.0, 11),
                 (0.0, float("inf"), 1.0, 11)):
        assert lib.tera_cell_thresholds(*args, p) == _lib.EINVAL, args
    assert lib.tera_cell_thresholds(0.0, 10.0, 1.0, 11, None) == _lib.EINVAL

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

"""The partition's classification tables (tera_axis_buckets) against the
oracle's classification rule (paper Sec. 2.1, "Aura Update"; Sec. 2.4.1).

The device answers an axis from the table only when its float32 estimate of
the coordinate lands in a bucket that holds an answer; that answer must be
the rule's for every such coordinate.  These tests emulate the device's
estimate in numpy float32 arithmetic (mantissa cut to 20 bits, then
(f - flo) * fs rounded to nearest, truncated) for coordinates at and within a
few ulps of every threshold value and every bucket edge, and for random
coordinates inside and around the domain, and compare each answered bucket
with the oracle's owner box and aura bits for that axis.  No GPU is needed.
"""
import math

import numpy as np
import pytest

from paper_2509_24063_gb300 import build

AXIS_BUCKETS = 8192
EXACT = 0x80
# mask bits of the offsets (-1, 0, 0), (+1, 0, 0), (0, -1, 0), ... (bit dx+1 + 3(dy+1) + 9(dz+1))
LOW_BIT = (12, 10, 4)
HIGH_BIT = (14, 16, 22)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def edges(lo, hi, n):
    e = [lo + ((hi - lo) * k) / n for k in range(n)]
    e.append(hi)
    return e


def device_buckets(v, flo, fs):
    """The bucket the device computes for each binary64 value (-1: no estimate
    or outside the table)."""
    bits = np.ascontiguousarray(v, dtype=np.float64).view(np.uint64)
    hi = (bits >> np.uint64(32)).astype(np.uint32)
    ha = hi & np.uint32(0x7FFFFFFF)
    ok = (ha - np.uint32(0x38100000)) < np.uint32(0x0FE00000)  # wraps like u32
    fbits = (hi & np.uint32(0x80000000)) | ((ha - np.uint32(0x38000000)) << np.uint32(3))
    af = fbits.view(np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        f = (af - np.float32(flo)) * np.float32(fs)
        assert f.dtype == np.float32
        j = np.where(np.isfinite(f) & (f > -1.0) & (f < AXIS_BUCKETS), np.trunc(f), -1)
    return np.where(ok, j, -1).astype(np.int64)


def ulp_walk(x, k):
    out = []
    y = x
    for _ in range(k):
        y = math.nextafter(y, -math.inf)
    for _ in range(2 * k + 1):
        out.append(y)
        y = math.nextafter(y, math.inf)
    return out


def axis_values(lo, hi, n, w, rng):
    """Coordinates of one axis: each threshold value and bucket edge with its
    3 ulp neighbours either side, and random values over [lo, hi) and a
    margin around it."""
    e = edges(lo, hi, n)
    th = [lo, hi] + e[1:-1] + [e[k] + w for k in range(n)] + [e[k + 1] - w for k in range(n)]
    vals = []
    for t in th:
        vals += ulp_walk(t, 3)
    s = AXIS_BUCKETS / (hi - lo)
    for j in range(AXIS_BUCKETS + 1):
        vals += ulp_walk(lo + j / s, 2)
    span = hi - lo
    vals += list(rng.uniform(lo - 0.05 * span, hi + 0.05 * span, 20000))
    return np.array(vals, dtype=np.float64)


def check_grid(oracle, lo, hi, n, w, periodic=0, seed=0, expect_tables=True):
    from paper_2509_24063_gb300.api import axis_buckets
    got = axis_buckets(lo, hi, n, w, periodic)
    if not expect_tables:
        assert got is None
        return 0
    assert got is not None
    tab, flo, fs = got
    grid = oracle.make_grid(lo, hi, n, w, periodic)
    rng = np.random.default_rng(seed)
    checked = 0
    for a in range(3):
        v = axis_values(lo[a], hi[a], n[a], w, rng)
        j = device_buckets(v, flo[a], fs[a])
        ent = np.where(j >= 0, tab[a][np.clip(j, 0, AXIS_BUCKETS - 1)], EXACT)
        answered = ent != EXACT
        v, ent = v[answered], ent[answered].astype(np.int64)
        if v.size == 0:
            continue
        # the other two coordinates at their domain's middle
        pts = [np.full(v.size, 0.5 * (lo[b] + hi[b])) for b in range(3)]
        pts[a] = v
        st, owner, mask = oracle.classify(grid, *pts)
        assert st == oracle.OK or st == oracle.EDOMAIN
        # an answered coordinate is inside the domain
        assert np.all(owner >= 0), v[owner < 0][:5]
        stride = [1, n[0], n[0] * n[1]][a]
        box = (owner.astype(np.int64) // stride) % n[a]
        low = (mask.astype(np.int64) >> LOW_BIT[a]) & 1
        high = (mask.astype(np.int64) >> HIGH_BIT[a]) & 1
        bad = (box != ent >> 2) | (low != (ent & 1)) | (high != ((ent >> 1) & 1))
        assert not bad.any(), (a, v[bad][:5], ent[bad][:5], box[bad][:5])
        checked += int(v.size)
    return checked


@pytest.mark.parametrize("name", ["uniform_1m", "blobs_16m", "uniform_100m", "torus_1m"])
def test_tables_of_the_workload_grids(libpath, oracle, name):
    import synth
    wl = synth.WORKLOADS[name]
    checked = check_grid(oracle, wl.lo, wl.hi, wl.grid, wl.w, wl.periodic, seed=1)
    assert checked > 50000


@pytest.mark.parametrize("seed", range(6))
def test_tables_of_random_grids(libpath, oracle, seed):
    rng = np.random.default_rng(100 + seed)
    n = [int(rng.integers(1, 33)) for _ in range(3)]
    periodic = int(rng.integers(0, 8))
    periodic &= sum(1 << a for a in range(3) if n[a] >= 3)
    lo = [float(rng.uniform(-2000, 2000)) for _ in range(3)]
    side = [float(rng.uniform(0.5, 300)) for _ in range(3)]
    hi = [lo[a] + side[a] * n[a] for a in range(3)]
    w = float(rng.uniform(0.05, 0.95)) * min(side)
    checked = check_grid(oracle, lo, hi, n, w, periodic, seed=seed)
    assert checked > 30000


def test_threshold_just_beside_a_bucket_edge(libpath, oracle):
    """Domain [-8192, 0) in 8 boxes: buckets of width 1, so every integer is a
    bucket edge on the estimate's grid.  With w = 30 + 2^-20 the aura threshold
    e[1] - w of box 0 lies 2^-20 below the edge -7198.  A value one ulp below
    the threshold has its mantissa cut toward zero, onto the edge, so the
    estimate places it in the bucket above the edge, which must not answer:
    the threshold lies within the estimate's error of that bucket."""
    w = 30.0 + 2.0 ** -20
    lo, hi, n = (-8192.0,) * 3, (0.0,) * 3, (8, 8, 8)
    t = (-8192.0 + 1024.0) - w
    assert -7198.0 - t == 2.0 ** -20
    checked = check_grid(oracle, lo, hi, n, w, 0, seed=11)
    assert checked > 50000
    from paper_2509_24063_gb300.api import axis_buckets
    tab, flo, fs = axis_buckets(lo, hi, n, w)
    v = np.array([math.nextafter(t, -math.inf)])
    j = int(device_buckets(v, flo[0], fs[0])[0])
    assert j == 994 and tab[0][j] == EXACT


def test_domain_across_zero(libpath, oracle):
    """Values near zero have no float estimate (|v| < 2^-126) or tiny ones: the
    exact comparisons decide there, and the answered buckets stay right."""
    checked = check_grid(oracle, (-10.0, -5.0, -1.0), (10.0, 7.0, 1.0), (4, 3, 2), 0.4, 0, seed=7)
    assert checked > 50000


@pytest.mark.parametrize("lo,hi,n,w", [
    ((0.0, 0.0, 0.0), (330.0, 10.0, 10.0), (33, 1, 1), 1.0),          # more than 32 boxes
    ((1.0e6, 0.0, 0.0), (1.0e6 + 3.0, 1.0, 1.0), (1, 1, 1), 0.01),    # estimate too coarse
])
def test_grids_without_tables(libpath, oracle, lo, hi, n, w):
    check_grid(oracle, lo, hi, n, w, expect_tables=False)


def test_axis_buckets_rejects_bad_grids(libpath):
    from paper_2509_24063_gb300 import _lib
    from paper_2509_24063_gb300.api import axis_buckets
    for lo, hi, n, w in [((0, 0, 0), (10, 10, 10), (0, 1, 1), 1.0),
                         ((0, 0, 0), (10, 10, 10), (2, 2, 2), 6.0),
                         ((0, 0, 0), (0, 10, 10), (1, 1, 1), 1.0)]:
        with pytest.raises(_lib.TeraError):
            axis_buckets(lo, hi, n, w)

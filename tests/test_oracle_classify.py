"""Pins for the oracle's grid classification (paper Sec. 2.1, "Aura Update").

The reference point is a brute force over ALL boxes of the grid: an agent is
sent to box b (b != owner) when it lies in b's region expanded by the aura
width w on every axis (L-infinity), e[b] - w <= v < e[b+1] + w.  This shares
nothing with the oracle's per-axis counting rule, so a wrong index, a dropped
neighbour-existence test, a swapped bit layout or a wrong owner formula fails.
"""
import itertools
import math

import numpy as np
import pytest


def edges(lo, hi, n):
    e = [lo + ((hi - lo) * k) / n for k in range(n)]
    e.append(hi)
    return e


def brute_force(grid_lo, grid_hi, grid_n, w, pts):
    E = [edges(grid_lo[a], grid_hi[a], grid_n[a]) for a in range(3)]
    owners, masks = [], []
    for v in pts:
        if not all(grid_lo[a] <= v[a] < grid_hi[a] for a in range(3)):
            owners.append(-1)
            masks.append(0)
            continue
        own = None
        inside = []
        for b in itertools.product(*(range(grid_n[a]) for a in range(3))):
            if all(E[a][b[a]] <= v[a] < E[a][b[a] + 1] for a in range(3)):
                assert own is None
                own = b
            if all(E[a][b[a]] - w <= v[a] < E[a][b[a] + 1] + w for a in range(3)):
                inside.append(b)
        assert own is not None
        m = 0
        for b in inside:
            if b == own:
                continue
            o = [b[a] - own[a] for a in range(3)]
            assert all(-1 <= t <= 1 for t in o)  # w < side: only direct neighbours
            m |= 1 << ((o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1))
        owners.append(own[0] + grid_n[0] * (own[1] + grid_n[1] * own[2]))
        masks.append(m)
    return np.array(owners, dtype=np.int32), np.array(masks, dtype=np.uint32)


def random_case(rng):
    n = [int(rng.integers(1, 4)) for _ in range(3)]
    lo = [float(rng.uniform(-50, 50)) for _ in range(3)]
    side = [float(rng.uniform(5, 40)) for _ in range(3)]
    hi = [lo[a] + side[a] * n[a] for a in range(3)]
    min_side = min(min(np.diff(edges(lo[a], hi[a], n[a]))) for a in range(3))
    w = float(rng.uniform(0.05, 0.999)) * min_side
    N = int(rng.integers(0, 257))
    pts = []
    E = [edges(lo[a], hi[a], n[a]) for a in range(3)]
    for _ in range(N):
        v = []
        for a in range(3):
            r = rng.random()
            if r < 0.15:  # exactly on an edge
                v.append(float(E[a][int(rng.integers(0, n[a]))]))
            elif r < 0.3:  # exactly on an aura threshold (inside the domain)
                k = int(rng.integers(0, n[a] + 1))
                t = E[a][k] + (w if rng.random() < 0.5 else -w)
                v.append(min(max(t, lo[a]), math.nextafter(hi[a], lo[a])))
            elif r < 0.35:  # one ulp around a threshold
                k = int(rng.integers(0, n[a] + 1))
                t = math.nextafter(E[a][k] + w, -math.inf if rng.random() < 0.5 else math.inf)
                v.append(min(max(t, lo[a]), math.nextafter(hi[a], lo[a])))
            else:
                v.append(float(rng.uniform(lo[a], hi[a])))
        pts.append(v)
    return lo, hi, n, w, pts


@pytest.mark.parametrize("seed", range(40))
def test_classify_matches_all_boxes_brute_force(oracle, seed):
    rng = np.random.default_rng(1000 + seed)
    lo, hi, n, w, pts = random_case(rng)
    g = oracle.make_grid(lo, hi, n, w)
    assert oracle.grid_check(g) == oracle.OK
    P = np.array(pts, dtype=np.float64).reshape(-1, 3)
    st, owner, mask = oracle.classify(g, P[:, 0], P[:, 1], P[:, 2])
    assert st == oracle.OK
    bo, bm = brute_force(lo, hi, n, w, pts)
    np.testing.assert_array_equal(owner, bo)
    np.testing.assert_array_equal(mask, bm)
    # conservation: every in-domain agent has exactly one owner box
    assert np.all(owner >= 0) and np.all(owner < n[0] * n[1] * n[2])
    # the self bit never appears
    assert np.all((mask >> 13) & 1 == 0)


def test_classify_hypothesis(oracle):
    hyp = pytest.importorskip("hypothesis")
    st_ = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None)
    @hyp.given(st_.integers(0, 2**32 - 1))
    def run(seed):
        rng = np.random.default_rng(seed)
        lo, hi, n, w, pts = random_case(rng)
        g = oracle.make_grid(lo, hi, n, w)
        P = np.array(pts, dtype=np.float64).reshape(-1, 3)
        s, owner, mask = oracle.classify(g, P[:, 0], P[:, 1], P[:, 2])
        bo, bm = brute_force(lo, hi, n, w, pts)
        assert s == oracle.OK
        assert np.array_equal(owner, bo) and np.array_equal(mask, bm)

    run()


def test_both_sides_of_one_axis_when_box_is_narrower_than_two_auras(oracle):
    # side 50, w 30: x in [20, 30) lies within w of both faces of box 0 of 2
    g = oracle.make_grid((0, 0, 0), (100, 100, 100), (2, 2, 1), 30.0)
    x = np.array([25.0, 55.0, 75.0]); y = np.array([10.0, 60.0, 50.0]); z = np.zeros(3)
    st, owner, mask = oracle.classify(g, x, y, z)
    assert st == oracle.OK
    # agent 0: box (0,0); x=25 -> +x neighbour only (x<30 would be -x but i=0);
    # y=10 -> +y? 10 >= 50-30 = 20 is false -> no.  So only bit (+1,0,0) = 14.
    assert owner[0] == 0 and mask[0] == 1 << 14
    # agent 1: box (1,1); x=55 < 50+30 -> -x; y=60 < 80 -> -y; corner too.
    assert owner[1] == 3
    assert mask[1] == (1 << 12) | (1 << 10) | (1 << 9)
    # agent 2: box (1,1); x=75 < 80 -> -x; y=50 -> -y (50 < 80); corner.
    assert owner[2] == 3 and mask[2] == (1 << 12) | (1 << 10) | (1 << 9)


def test_domain_errors(oracle):
    g = oracle.make_grid((0, 0, 0), (10, 10, 10), (2, 2, 2), 1.0)
    x = np.array([0.0, 10.0, -1e-300, np.nan, 9.999, 5.0])
    y = np.array([0.0, 1.0, 1.0, 1.0, 1.0, np.inf])
    z = np.zeros(6)
    st, owner, mask = oracle.classify(g, x, y, z)
    assert st == oracle.EDOMAIN
    np.testing.assert_array_equal(owner, [0, -1, -1, -1, 1, -1])
    assert mask[1] == mask[2] == mask[3] == mask[5] == 0


@pytest.mark.parametrize("w,ok", [(0.0, False), (-1.0, False), (5.0, False), (4.999, True),
                                  (np.nan, False)])
def test_grid_check_aura_narrower_than_box(oracle, w, ok):
    g = oracle.make_grid((0, 0, 0), (10, 10, 10), (2, 2, 2), w)
    assert (oracle.grid_check(g) == oracle.OK) == ok


def test_edges_definition(oracle):
    g = oracle.make_grid((0.1, -3.0, 7.0), (0.7, 5.0, 7.3), (3, 7, 1), 0.01)
    for a, (lo, hi, n) in enumerate([(0.1, 0.7, 3), (-3.0, 5.0, 7), (7.0, 7.3, 1)]):
        assert list(oracle.axis_edges(g, a)) == edges(lo, hi, n)
        assert oracle.axis_edges(g, a)[-1] == hi


# ---- toroidal axes (Sec. 2.5 names open, closed and toroidal boundaries) ----
# On a periodic axis the region of box b expanded by w wraps round the domain:
# box n-1 also covers [lo, e[0] + w) and box 0 also covers [e[n] - w, hi).  The
# offset of box b seen from the owner is (b - own) taken modulo n into
# {-1, 0, +1}, unique because a periodic axis has at least 3 boxes.

def brute_force_periodic(grid_lo, grid_hi, grid_n, w, periodic, pts):
    E = [edges(grid_lo[a], grid_hi[a], grid_n[a]) for a in range(3)]

    def covers(a, b, v):
        n = grid_n[a]
        if E[a][b] - w <= v < E[a][b + 1] + w:
            return True
        if periodic >> a & 1:
            if b == n - 1 and v < E[a][0] + w:
                return True
            if b == 0 and v >= E[a][n] - w:
                return True
        return False

    owners, masks = [], []
    for v in pts:
        own = None
        inside = []
        for b in itertools.product(*(range(grid_n[a]) for a in range(3))):
            if all(E[a][b[a]] <= v[a] < E[a][b[a] + 1] for a in range(3)):
                assert own is None
                own = b
            if all(covers(a, b[a], v[a]) for a in range(3)):
                inside.append(b)
        assert own is not None
        m = 0
        for b in inside:
            if b == own:
                continue
            o = []
            for a in range(3):
                d = b[a] - own[a]
                if periodic >> a & 1:
                    d = (d + 1) % grid_n[a] - 1
                assert -1 <= d <= 1
                o.append(d)
            m |= 1 << ((o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1))
        owners.append(own[0] + grid_n[0] * (own[1] + grid_n[1] * own[2]))
        masks.append(m)
    return np.array(owners, dtype=np.int32), np.array(masks, dtype=np.uint32)


def random_periodic_case(rng):
    periodic = int(rng.integers(1, 8))
    lo, hi, n, w, _ = random_case(rng)
    n = [int(rng.integers(3, 6)) if periodic >> a & 1 else n[a] for a in range(3)]
    min_side = min(min(np.diff(edges(lo[a], hi[a], n[a]))) for a in range(3))
    w = float(rng.uniform(0.05, 0.999)) * min_side
    E = [edges(lo[a], hi[a], n[a]) for a in range(3)]
    pts = []
    for _ in range(int(rng.integers(0, 257))):
        v = []
        for a in range(3):
            r = rng.random()
            if r < 0.3:  # on a threshold, the wrap-round ones included
                k = int(rng.integers(0, n[a] + 1))
                t = E[a][k] + (w if rng.random() < 0.5 else -w)
                v.append(min(max(t, lo[a]), math.nextafter(hi[a], lo[a])))
            elif r < 0.4:  # within w of the domain faces
                t = lo[a] + w * rng.random() if rng.random() < 0.5 else hi[a] - w * rng.random()
                v.append(min(max(t, lo[a]), math.nextafter(hi[a], lo[a])))
            elif r < 0.45:
                v.append(lo[a] if rng.random() < 0.5 else math.nextafter(hi[a], lo[a]))
            else:
                v.append(float(rng.uniform(lo[a], hi[a])))
        pts.append(v)
    return lo, hi, n, w, periodic, pts


@pytest.mark.parametrize("seed", range(40))
def test_classify_periodic_matches_wrapped_brute_force(oracle, seed):
    rng = np.random.default_rng(5000 + seed)
    lo, hi, n, w, periodic, pts = random_periodic_case(rng)
    g = oracle.make_grid(lo, hi, n, w, periodic)
    assert oracle.grid_check(g) == oracle.OK
    P = np.array(pts, dtype=np.float64).reshape(-1, 3)
    st, owner, mask = oracle.classify(g, P[:, 0], P[:, 1], P[:, 2])
    assert st == oracle.OK
    bo, bm = brute_force_periodic(lo, hi, n, w, periodic, pts)
    np.testing.assert_array_equal(owner, bo)
    np.testing.assert_array_equal(mask, bm)


def test_periodic_hand_example(oracle):
    # 90^3 cube, 3x3x3 boxes of side 30, w 10, only x wraps
    g = oracle.make_grid((0, 0, 0), (90, 90, 90), (3, 3, 3), 10.0, periodic=1)
    x = np.array([5.0, 85.0, 5.0, 45.0])
    y = np.array([45.0, 45.0, 5.0, 45.0])
    z = np.array([45.0, 45.0, 45.0, 45.0])
    st, owner, mask = oracle.classify(g, x, y, z)
    assert st == oracle.OK
    # x = 5 in box 0: the -x neighbour is box 2 across the boundary, bit 12
    assert owner[0] == 0 + 3 * (1 + 3 * 1) and mask[0] == 1 << 12
    # x = 85 in box 2: the +x neighbour is box 0, bit 14
    assert owner[1] == 2 + 3 * (1 + 3 * 1) and mask[1] == 1 << 14
    # y = 5 does not wrap (y closed): only -x (bit 12); no -y or corner bits
    assert mask[2] == 1 << 12
    # the middle of the middle box sends nothing
    assert mask[3] == 0
    # the same agents on a closed grid lose the wrap-round bits
    gc = oracle.make_grid((0, 0, 0), (90, 90, 90), (3, 3, 3), 10.0)
    st, owner_c, mask_c = oracle.classify(gc, x, y, z)
    np.testing.assert_array_equal(owner_c, owner)
    assert list(mask_c) == [0, 0, 0, 0]


@pytest.mark.parametrize("n,periodic,reserved,ok", [
    ((3, 3, 3), 7, 0, True), ((2, 3, 3), 1, 0, False), ((2, 3, 3), 6, 0, True),
    ((3, 3, 1), 4, 0, False), ((3, 3, 3), 8, 0, False), ((3, 3, 3), 0, 1, False)])
def test_grid_check_periodic(oracle, n, periodic, reserved, ok):
    g = oracle.make_grid((0, 0, 0), (30, 30, 30), n, 1.0, periodic)
    g.reserved = reserved
    assert (oracle.grid_check(g) == oracle.OK) == ok


def test_threaded_classification_equals_single_threaded(oracle):
    rng = np.random.default_rng(4)
    g = oracle.make_grid((0, 0, 0), (100, 80, 60), (5, 4, 3), 6.0)
    n = 300001
    x, y, z = rng.uniform(0, 100, n), rng.uniform(0, 80, n), rng.uniform(0, 60, n)
    x[17] = np.nan  # an agent outside the domain, in the first range
    a = oracle.classify(g, x, y, z)
    b = oracle.classify(g, x, y, z, threads=6)
    assert a[0] == b[0] == oracle.EDOMAIN
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])

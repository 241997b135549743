"""Pins for the oracle's agent migration (paper Sec. 2.1 "Agent Migration";
records are the raw TeraAgent IO buffers of Sec. 2.2.1).

References that share nothing with the oracle's counting loops:
  * the definition restated as one sort: the next state of box d is its
    stayers in previous order, then its immigrants ordered by the side they
    arrive from (computed here from box coordinates) and then by index;
  * special cases: nothing moves (the state is unchanged, every inbox empty);
    every agent starts in box 0 (the result is numpy's stable argsort by owner);
  * invariants: a permutation of the records, every agent of box d owned by d;
  * hand-worked moves on a 3-box axis, closed and toroidal, and a far move.
"""
import math

import numpy as np
import pytest

COLS = ("x", "y", "z", "diameter", "volume", "adherence", "density")


def owners(oracle, g, st):
    s, o, _ = oracle.classify(g, st["x"], st["y"], st["z"])
    assert s == oracle.OK
    return o


def box_major(oracle, g, st):
    """Reorder a state by owner box (stable) and return it with its box offsets."""
    o = owners(oracle, g, st)
    perm = np.argsort(o, kind="stable")
    nb = int(g.n[0] * g.n[1] * g.n[2])
    out = {k: np.ascontiguousarray(v[perm]) for k, v in st.items()}
    off = np.zeros(nb + 1, dtype=np.uint64)
    off[1:] = np.cumsum(np.bincount(o, minlength=nb))
    return out, off


def random_state(rng, n, lo, hi):
    st = {"id": rng.permutation(n).astype(np.uint64)}
    for a, k in enumerate("xyz"):
        st[k] = rng.uniform(lo[a], hi[a], n)
    for k in ("diameter", "volume", "adherence", "density"):
        st[k] = rng.uniform(0.5, 2.0, n)
    return st


def move(rng, st, lo, hi, sigma, periodic, p_far=0.0):
    st = {k: v.copy() for k, v in st.items()}
    n = st["x"].shape[0]
    far = rng.random(n) < p_far
    for a, k in enumerate("xyz"):
        v = st[k] + sigma * rng.standard_normal(n)
        v = np.where(far, rng.uniform(lo[a], hi[a], n), v)
        L = hi[a] - lo[a]
        if periodic >> a & 1:
            v = lo[a] + np.mod(v - lo[a], L)
        v = np.minimum(np.maximum(v, lo[a]), math.nextafter(hi[a], lo[a]))
        st[k] = v
    return st


def side(grid_n, periodic, s, d):
    """Neighbour bit of the offset from box d to box s, 13 when not neighbours."""
    def coords(b):
        return (b % grid_n[0], (b // grid_n[0]) % grid_n[1], b // (grid_n[0] * grid_n[1]))
    cs, cd = coords(s), coords(d)
    o = []
    for a in range(3):
        t = cs[a] - cd[a]
        if periodic >> a & 1:
            t = (t + 1) % grid_n[a] - 1
        if abs(t) > 1:
            return 13
        o.append(t)
    return (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1)


def expected(oracle, g, grid_n, periodic, st, box_off):
    n = st["x"].shape[0]
    nb = grid_n[0] * grid_n[1] * grid_n[2]
    src = np.repeat(np.arange(nb), np.diff(box_off.astype(np.int64)))
    dst = owners(oracle, g, st)
    keys = []
    for i in range(n):
        s, d = int(src[i]), int(dst[i])
        b = -1 if s == d else side(grid_n, periodic, s, d)
        keys.append((d, b, i))
    order = [k[2] for k in sorted(keys)]
    return np.array(order, dtype=np.int64), src, dst


def check_against_definition(oracle, lo, hi, grid_n, w, periodic, st, box_off):
    g = oracle.make_grid(lo, hi, grid_n, w, periodic)
    res = oracle.migrate(g, st, box_off)
    assert res["status"] == oracle.OK
    order, src, dst = expected(oracle, g, grid_n, periodic, st, box_off)
    nxt = res["next"]
    for k in ("id",) + COLS:
        np.testing.assert_array_equal(nxt[k].view(np.uint64), st[k][order].view(np.uint64))
    nb = grid_n[0] * grid_n[1] * grid_n[2]
    np.testing.assert_array_equal(res["box_off_next"][1:],
                                  np.cumsum(np.bincount(dst, minlength=nb)))
    # each inbox holds its leavers in agent order, as raw records after a header
    Q = nb * 27
    off = res["inbox_off"]
    arena = res["arena"]
    for q in range(Q):
        d, b = divmod(q, 27)
        members = [i for i in range(len(src))
                   if dst[i] == d and src[i] != d and side(grid_n, periodic, src[i], d) == b]
        assert int(off[q + 1] - off[q]) == len(members)
        h = arena[(int(off[q]) + q) * 64:(int(off[q]) + q + 1) * 64]
        assert h[:4].tobytes() == b"TAIO" and int(h[12:16].view(np.uint32)[0]) == q
        assert int(h[16:24].view(np.uint64)[0]) == len(members)
        recs = arena[(int(off[q]) + q + 1) * 64:(int(off[q + 1]) + q + 1) * 64].view(np.uint64)
        recs = recs.reshape(-1, 8)
        for r, i in zip(recs, members):
            assert r[0] == st["id"][i]
            for c, k in enumerate(COLS):
                assert r[c + 1] == st[k][i:i + 1].view(np.uint64)[0]
    return res


@pytest.mark.parametrize("seed", range(12))
def test_migration_matches_definition(oracle, seed):
    rng = np.random.default_rng(7000 + seed)
    periodic = int(rng.integers(0, 8))
    grid_n = [int(rng.integers(3, 5)) if periodic >> a & 1 else int(rng.integers(1, 4))
              for a in range(3)]
    lo = [float(rng.uniform(-20, 20)) for _ in range(3)]
    hi = [lo[a] + 10.0 * grid_n[a] for a in range(3)]
    n = int(rng.integers(0, 300))
    g = oracle.make_grid(lo, hi, grid_n, 1.0, periodic)
    st0, off = box_major(oracle, g, random_state(rng, n, lo, hi))
    st1 = move(rng, st0, lo, hi, sigma=float(rng.uniform(0.5, 6.0)), periodic=periodic,
               p_far=0.05)
    check_against_definition(oracle, lo, hi, grid_n, 1.0, periodic, st1, off)


def test_nothing_moves(oracle):
    rng = np.random.default_rng(3)
    lo, hi, grid_n = (0, 0, 0), (30, 30, 30), (3, 3, 3)
    g = oracle.make_grid(lo, hi, grid_n, 1.0)
    st, off = box_major(oracle, g, random_state(rng, 500, lo, hi))
    res = oracle.migrate(g, st, off)
    assert res["status"] == oracle.OK
    assert int(res["inbox_off"][-1]) == 0
    np.testing.assert_array_equal(res["box_off_next"], off)
    for k in ("id",) + COLS:
        np.testing.assert_array_equal(res["next"][k], st[k])


@pytest.mark.parametrize("periodic", [0, 7])
def test_regroup_from_box_zero_is_stable_sort_by_owner(oracle, periodic):
    rng = np.random.default_rng(4 + periodic)
    lo, hi, grid_n = (0, 0, 0), (40, 30, 30), (4, 3, 3)
    g = oracle.make_grid(lo, hi, grid_n, 1.0, periodic)
    st = random_state(rng, 700, lo, hi)
    nb = 36
    off = np.full(nb + 1, 700, dtype=np.uint64)
    off[0] = 0
    res = oracle.migrate(g, st, off)
    assert res["status"] == oracle.OK
    o = owners(oracle, g, st)
    perm = np.argsort(o, kind="stable")
    for k in ("id",) + COLS:
        np.testing.assert_array_equal(res["next"][k], st[k][perm])


def hand_state(xs):
    n = len(xs)
    return {"id": np.arange(100, 100 + n, dtype=np.uint64), "x": np.array(xs, dtype=np.float64),
            "y": np.full(n, 5.0), "z": np.full(n, 5.0), "diameter": np.arange(n, dtype=np.float64),
            "volume": np.ones(n), "adherence": np.ones(n), "density": np.ones(n)}


def test_hand_moves_closed_axis(oracle):
    # three boxes of side 10 along x; previous boxes [0, 0, 1, 1, 2]
    g = oracle.make_grid((0, 0, 0), (30, 10, 10), (3, 1, 1), 1.0)
    st = hand_state([12.0, 3.0, 8.0, 15.0, 25.0])  # agent 0 left box 0 for box 1, agent 2 box 1 -> 0
    off = np.array([0, 2, 4, 5], dtype=np.uint64)
    res = oracle.migrate(g, st, off)
    assert res["status"] == oracle.OK
    # box 0: stayer 1, then agent 2 arriving from +x (side 14)
    # box 1: stayer 3, then agent 0 arriving from -x (side 12); box 2: agent 4
    assert list(res["next"]["id"]) == [101, 102, 103, 100, 104]
    assert list(res["box_off_next"]) == [0, 2, 4, 5]
    inbox = res["inbox_off"]
    assert int(inbox[0 * 27 + 15] - inbox[0 * 27 + 14]) == 1   # box 0, from +x
    assert int(inbox[1 * 27 + 13] - inbox[1 * 27 + 12]) == 1   # box 1, from -x
    assert int(inbox[-1]) == 2


def test_hand_far_move_and_wrap(oracle):
    st = hand_state([25.0, 5.0])  # agent 0 was in box 0 and is now in box 2
    off = np.array([0, 2, 2, 2], dtype=np.uint64)
    g = oracle.make_grid((0, 0, 0), (30, 10, 10), (3, 1, 1), 1.0)
    res = oracle.migrate(g, st, off)
    inbox = res["inbox_off"]
    # closed axis: box 0 is not a neighbour of box 2, side 13
    assert int(inbox[2 * 27 + 14] - inbox[2 * 27 + 13]) == 1
    gp = oracle.make_grid((0, 0, 0), (30, 10, 10), (3, 1, 1), 1.0, periodic=1)
    res = oracle.migrate(gp, st, off)
    inbox = res["inbox_off"]
    # toroidal axis: box 0 is the +x neighbour of box 2, side 14
    assert int(inbox[2 * 27 + 15] - inbox[2 * 27 + 14]) == 1
    assert list(res["next"]["id"]) == [101, 100]


def test_errors(oracle):
    g = oracle.make_grid((0, 0, 0), (30, 10, 10), (3, 1, 1), 1.0)
    st = hand_state([12.0, 3.0, 8.0, 15.0, 25.0])
    for bad in ([0, 2, 4, 6], [1, 2, 4, 5], [0, 3, 2, 5]):
        assert oracle.migrate(g, st, np.array(bad, dtype=np.uint64))["status"] == oracle.EINVAL
    off = np.array([0, 2, 4, 5], dtype=np.uint64)
    # 81 inbox headers + 2 records do not fit in 82 units
    assert oracle.migrate(g, st, off, arena_units=82)["status"] == oracle.ECAPACITY
    assert oracle.migrate(g, st, off, arena_units=83)["status"] == oracle.OK
    st_bad = hand_state([12.0, 3.0, 8.0, 30.0, 25.0])
    assert oracle.migrate(g, st_bad, off)["status"] == oracle.EDOMAIN
    # a damaged inbox header is refused by the receiver
    res = oracle.migrate(g, st, off)
    arena = res["arena"].copy()
    q = 1 * 27 + 12
    arena[(int(res["inbox_off"][q]) + q) * 64 + 16] ^= 1
    nxt = {k: np.zeros_like(v) for k, v in res["next"].items()}
    assert oracle.migrate_recv(g, arena, res["inbox_off"], res["box_off_next"], nxt) == \
        oracle.ECORRUPT


def test_invariants_larger(oracle):
    rng = np.random.default_rng(11)
    lo, hi, grid_n = (0, 0, 0), (100, 100, 100), (4, 4, 4)
    g = oracle.make_grid(lo, hi, grid_n, 5.0)
    st0, off = box_major(oracle, g, random_state(rng, 20000, lo, hi))
    st1 = move(rng, st0, lo, hi, sigma=3.0, periodic=0, p_far=0.01)
    res = oracle.migrate(g, st1, off)
    assert res["status"] == oracle.OK
    nxt, bo = res["next"], res["box_off_next"]
    np.testing.assert_array_equal(np.sort(nxt["id"]), np.sort(st1["id"]))
    o = owners(oracle, g, nxt)
    np.testing.assert_array_equal(o, np.repeat(np.arange(64), np.diff(bo.astype(np.int64))))
    # stayers keep their relative order inside each box
    src = np.repeat(np.arange(64), np.diff(off.astype(np.int64)))
    o1 = owners(oracle, g, st1)
    for d in range(64):
        stay_ids = st1["id"][(src == d) & (o1 == d)]
        a = int(bo[d])
        np.testing.assert_array_equal(nxt["id"][a:a + len(stay_ids)], stay_ids)

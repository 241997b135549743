"""Boxes sharded over ranks (paper Sec. 2.1; Sec. 2.4 "Load Balancing"): the
box-to-rank map, the diffusive rebalancing, and the routing of aura messages
and migration inboxes between ranks, on CPU.

The routing runs over two (or three) gloo ranks in separate processes; each
rank encodes, decodes and migrates with the oracle in place of the library's
kernels (the same arenas and messages), and what every rank ends with is
compared byte for byte with the single-rank oracle on the whole state."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_24063_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ---------------- geometry and the box map ----------------

@pytest.mark.parametrize("n,periodic", [((3, 2, 2), 0), ((4, 3, 3), 0), ((3, 3, 4), 5),
                                        ((3, 4, 3), 7)])
def test_pair_receivers_against_the_oracle_arrival_side(oracle, n, periodic):
    # pair p = s*27 + b sends towards the box at offset b; seen from that box,
    # s lies at the opposite offset: the oracle's migration side rule
    g = oracle.make_grid((0, 0, 0), (10.0 * n[0], 10.0 * n[1], 10.0 * n[2]), n, 1.0, periodic)
    d = shard.pair_receivers(n, periodic)
    B = n[0] * n[1] * n[2]
    for s in range(B):
        for b in range(27):
            r = int(d[s * 27 + b])
            if b == 13:
                assert r == -1
            elif r >= 0:
                assert oracle.inbox_bit(g, s, r) == 26 - b
            else:
                # no neighbour there: every box that is adjacent to s is reached by another bit
                assert all(oracle.inbox_bit(g, s, x) != 26 - b for x in range(B) if x != s)


def test_slab_owners_are_contiguous_and_balanced():
    for B, world in ((64, 2), (64, 3), (512, 8), (10, 4)):
        o = shard.slab_owners(B, world)
        assert np.all(np.diff(o) >= 0) and o[0] == 0 and o[-1] == world - 1
        counts = np.bincount(o, minlength=world)
        assert counts.max() - counts.min() <= 1
    w = np.array([10.0] + [1.0] * 19)  # one heavy box
    o = shard.slab_owners(20, 2, w)
    assert np.all(np.diff(o) >= 0)
    assert abs(w[o == 0].sum() - w[o == 1].sum()) <= 10.0


def test_diffusive_rebalance_moves_boundary_boxes_to_a_faster_neighbour():
    n = (4, 4, 1)
    owner = shard.slab_owners(16, 2)  # rank 0: boxes 0..7 (rows 0-1), rank 1: 8..15
    cost = np.ones(16)
    same = shard.diffusive_rebalance(owner, cost, [1.0, 1.0], n)
    assert np.array_equal(same, owner)  # balanced: nothing moves
    new = shard.diffusive_rebalance(owner, cost, [3.0, 1.0], n)
    moved = np.nonzero(new != owner)[0]
    assert moved.size > 0
    assert np.all(owner[moved] == 0) and np.all(new[moved] == 1)
    for k in moved:  # every moved box touched rank 1's region
        assert np.any(owner[shard.adjacent_boxes(n, 0, int(k))] == 1)
    # the moved time fits the gap to the average: 3 - 2 = 1 s, boxes of 3/8 s
    assert moved.size * 3.0 / 8.0 <= 1.0 + 1e-12
    assert np.count_nonzero(new == 0) >= 1


def test_diffusive_rebalance_converges_on_a_cost_model():
    # runtime proportional to the agents a rank holds; rounds of rebalancing
    # bring the slowest rank towards the mean
    rng = np.random.default_rng(2)
    n = (8, 8, 2)
    B = 128
    cost = rng.gamma(0.7, 1.0, B)
    cost[:20] *= 6.0  # a dense corner
    owner = shard.slab_owners(B, 4)

    def times(o):
        return np.array([cost[o == r].sum() for r in range(4)])
    t0 = times(owner)
    for _ in range(12):
        owner = shard.diffusive_rebalance(owner, cost, times(owner), n)
    t1 = times(owner)
    assert t1.max() / t1.mean() < t0.max() / t0.mean()
    assert sorted(np.unique(owner).tolist()) == [0, 1, 2, 3]


def test_pairs_to_reset_touch_a_moved_box():
    n = (3, 2, 2)
    old = shard.slab_owners(12, 2)
    new = old.copy()
    new[5] = 1 - new[5]
    p = shard.pairs_to_reset(old, new, n)
    d = shard.pair_receivers(n)
    assert p.size > 0
    for q in p:
        assert q // 27 == 5 or d[q] == 5
    for q in np.setdiff1d(np.nonzero(d >= 0)[0], p):
        assert q // 27 != 5 and d[q] != 5


# ---------------- ranks on gloo ----------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run(fn, world, *args):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_entry, args=(fn, r, world, port, out) + args)
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    for r, p in enumerate(procs):
        assert p.exitcode == 0, out.get(r)
    for r in range(world):
        assert out.get(r) == "ok", out.get(r)


def _entry(fn, rank, world, port, out, *args):
    import sys
    import traceback
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                                world_size=world)
        globals()[fn](rank, world, *args)
        dist.barrier()
        dist.destroy_process_group()
        out[rank] = "ok"
    except Exception:
        out[rank] = traceback.format_exc()
        raise


AURA_WL = dict(n0=30000, lo=(0.0,) * 3, hi=(200.0, 150.0, 150.0), grid=(4, 3, 3), w=15.0)


def _aura_ranks(rank, world):
    import oracle
    from synth import Generator, Workload, to_numpy
    wl = Workload("t", AURA_WL["n0"], AURA_WL["lo"], AURA_WL["hi"], AURA_WL["grid"],
                  AURA_WL["w"], 4, p_grow=0.1, p_divide=0.02, p_die=0.02, seed=41)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    P = oracle.n_pairs(g)
    B = P // 27
    tr = shard.DistTransport()
    owner = shard.slab_owners(B, world)
    prev_g = prev_l = None  # single-rank and this rank's ((sender ref), (receiver ref))
    for t, st in enumerate(Generator(wl).series(4)):
        s = to_numpy(st)
        reset = np.zeros(P, dtype=np.uint8)
        if t == 2:  # the first rank is slower: boxes move, their pairs are sent raw once
            new = shard.diffusive_rebalance(owner, np.ones(B), [2.0] + [1.0] * (world - 1),
                                            wl.grid)
            assert np.count_nonzero(new != owner) > 0
            reset[shard.pairs_to_reset(owner, new, wl.grid)] = 1
            owner = new
        plan = shard.WirePlan(owner, wl.grid, 0, rank, world)
        # the whole state on one rank (the reference)
        _, own_b, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        _, _, off, idx = oracle.pair_lists(g, own_b, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro = (None, None) if prev_g is None else prev_g[0]
        st_, wire, wo, wlen, nxt = oracle.encode_all(rec, off, ra, ro, reset=reset)
        assert st_ == oracle.OK
        va, vo = (None, None) if prev_g is None else prev_g[1]
        st_, recv, roff = oracle.decode_all(wire, wo, va, vo)
        assert st_ == oracle.OK
        # this rank: the agents of its boxes, in their order
        keep = owner[own_b] == rank
        sl = {k: np.ascontiguousarray(v[keep]) for k, v in s.items()}
        _, ob, mk = oracle.classify(g, sl["x"], sl["y"], sl["z"])
        _, _, loff, lidx = oracle.pair_lists(g, ob, mk)
        lrec = oracle.pack(sl, loff, lidx)
        la, lo = (None, None) if prev_l is None else prev_l[0]
        lreset = reset * (owner[np.arange(P) // 27] == rank)
        st_, lwire, lwo, lwl, lnxt = oracle.encode_all(lrec, loff, la, lo, reset=lreset)
        assert st_ == oracle.OK
        local = (torch.from_numpy(lwire), torch.from_numpy(lwo.view(np.int64)),
                 torch.from_numpy(lwl.view(np.int64)))
        wire_in, off_in = shard.route_wire(plan, tr, local, 1, torch.device("cpu"))
        lv, lvo = (None, None) if prev_l is None else prev_l[1]
        st_, lrecv, lroff = oracle.decode_all(wire_in.numpy(), off_in.numpy().view(np.uint64),
                                              lv, lvo)
        assert st_ == oracle.OK
        # every pair this rank sends: message and new sender reference as on one rank
        sends = np.nonzero(owner[np.arange(P) // 27] == rank)[0]
        for p in sends:
            a, b = int(lwo[p]), int(lwo[p]) + int(lwl[p])
            ga = int(wo[p])
            assert lwire[a:b].tobytes() == wire[ga:ga + int(wlen[p])].tobytes(), (t, p)
            assert (oracle.arena_pair(lnxt, loff, p).tobytes()
                    == oracle.arena_pair(nxt, off, p).tobytes())
        # every pair this rank receives: the receive buffer as on one rank
        for p in plan.mine:
            assert (oracle.arena_pair(lrecv, lroff, p).tobytes()
                    == oracle.arena_pair(recv, roff, p).tobytes()), (t, p)
        # the pairs of other ranks' boxes decode to nothing here
        others = np.setdiff1d(np.arange(P), plan.mine)
        assert np.all(lroff[others + 1] == lroff[others])
        prev_g = ((nxt, off), (recv, roff))
        prev_l = ((lnxt, loff), (lrecv, lroff))


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_aura_exchange_equals_one_rank(world):
    _run("_aura_ranks", world)


def _migration_ranks(rank, world):
    import oracle
    from synth import Generator, Workload, to_numpy
    wl = Workload("t", 40000, (0.0,) * 3, (120.0, 120.0, 80.0), (4, 3, 2), 10.0, 2, seed=43)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    B = oracle.n_pairs(g) // 27
    s0, s1 = (to_numpy(x) for x in Generator(wl).series(2))
    # box-major state of the first positions, then the second positions
    _, own, _ = oracle.classify(g, s0["x"], s0["y"], s0["z"])
    perm = np.argsort(own, kind="stable")
    box_off = np.zeros(B + 1, dtype=np.uint64)
    box_off[1:] = np.cumsum(np.bincount(own, minlength=B))
    moved = {k: np.ascontiguousarray((s1 if k in ("x", "y", "z") else s0)[k][perm]) for k in s0}
    rng = np.random.default_rng(5)
    far = rng.choice(moved["x"].shape[0], 300, replace=False)  # moves far away (side 13)
    for a, k in enumerate(("x", "y", "z")):
        moved[k][far] = rng.uniform(wl.lo[a], wl.hi[a], far.size)
    ref = oracle.migrate(g, moved, box_off)
    assert ref["status"] == oracle.OK
    owner = shard.slab_owners(B, world)
    # this rank's part of the box-major state (empty boxes elsewhere)
    mine = owner == rank
    cnt = np.diff(box_off.astype(np.int64))
    lcnt = np.where(mine, cnt, 0)
    loff = np.zeros(B + 1, dtype=np.uint64)
    loff[1:] = np.cumsum(lcnt)
    sel = np.concatenate([np.arange(box_off[k], box_off[k + 1]) for k in np.nonzero(mine)[0]]
                         ).astype(np.int64)
    local = {k: np.ascontiguousarray(v[sel]) for k, v in moved.items()}
    res = oracle.migrate(g, local, loff)
    assert res["status"] == oracle.OK
    plan = shard.InboxPlan(owner, rank, world)
    own_t = (torch.from_numpy(res["arena"]), torch.from_numpy(res["inbox_off"].view(np.int64)))
    arena, inbox_off = shard.route_inboxes(plan, shard.DistTransport(), own_t, 1,
                                           torch.device("cpu"))
    final, src, dst = shard.stayer_layout(torch.from_numpy(res["box_off_next"].view(np.int64)),
                                          own_t[1], inbox_off)
    n = int(final[-1])
    nxt = {k: np.zeros(n, dtype=v.dtype) for k, v in res["next"].items()}
    for k in nxt:
        nxt[k][dst.numpy()] = res["next"][k][src.numpy()]
    code = oracle.migrate_recv(g, arena.numpy(), inbox_off.numpy().view(np.uint64),
                               final.numpy().view(np.uint64), nxt)
    assert code == oracle.OK
    gb = ref["box_off_next"].astype(np.int64)
    fb = final.numpy()
    for k in np.nonzero(mine)[0]:
        a, b = int(gb[k]), int(gb[k + 1])
        c, d = int(fb[k]), int(fb[k + 1])
        assert b - a == d - c, k
        for f in nxt:
            assert nxt[f][c:d].tobytes() == ref["next"][f][a:b].tobytes(), (k, f)
    for k in np.nonzero(~mine)[0]:
        assert fb[k + 1] == fb[k]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_migration_equals_one_rank(world):
    _run("_migration_ranks", world)


def _transfer_ranks(rank, world):
    rng = np.random.default_rng(11)
    n = (4, 4, 1)
    B = 16
    counts = rng.integers(0, 50, B)
    off = np.zeros(B + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    whole = {"id": np.arange(int(off[-1]), dtype=np.int64),
             "x": rng.standard_normal(int(off[-1]))}
    old = shard.slab_owners(B, world)
    new = shard.diffusive_rebalance(old, counts.astype(float) + 1.0,
                                    [3.0] + [1.0] * (world - 1), n)
    assert np.count_nonzero(new != old) > 0

    def part(owner):
        lc = np.where(owner == rank, counts, 0)
        lo = np.zeros(B + 1, dtype=np.int64)
        lo[1:] = np.cumsum(lc)
        sel = np.concatenate([np.arange(off[k], off[k + 1]) for k in range(B) if owner[k] == rank]
                             + [np.zeros(0, dtype=np.int64)]).astype(np.int64)
        return {k: torch.from_numpy(v[sel]) for k, v in whole.items()}, torch.from_numpy(lo)
    st, lo = part(old)
    got, got_off = shard.transfer_boxes(st, lo, old, new, rank, shard.DistTransport(),
                                        torch.device("cpu"))
    want, want_off = part(new)
    assert torch.equal(got_off, want_off)
    for k in want:
        assert torch.equal(got[k], want[k])


@pytest.mark.parametrize("world", [2, 3])
def test_box_transfer_after_rebalance(world):
    _run("_transfer_ranks", world)

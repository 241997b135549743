"""The sharded aura exchange and migration through the library's kernels, with
the ranks of a box map emulated in one process on one GPU: every rank's
kernels run one after another (no kernel waits for another rank), and the
buffers each rank would send are handed to the receiving rank's phase.  What
every rank ends with is compared byte for byte with the single-rank oracle."""
import numpy as np
import pytest
import torch

import oracle
from synth import Generator, Workload, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_exchange_ranks_match_one_rank(world):
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import shard
    wl = Workload("t", 60000, (0.0,) * 3, (200.0, 150.0, 150.0), (4, 3, 3), 15.0, 4,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=41)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    P = oracle.n_pairs(g)
    B = P // 27
    owner = shard.slab_owners(B, world)
    ctxs = [tera.Context(wl.lo, wl.hi, wl.grid, wl.w) for _ in range(world)]
    sx = [shard.ShardedExchange(ctxs[r], owner, r, world, 80000, 200000) for r in range(world)]
    prev = None
    for t, full in enumerate(Generator(wl, device="cuda").series(4)):
        st = {f: full[f] for f in FIELDS}
        s = to_numpy(st)
        reset = np.zeros(P, dtype=np.uint8)
        if t == 2:
            new = shard.diffusive_rebalance(owner, np.ones(B), [2.0] + [1.0] * (world - 1),
                                            wl.grid)
            assert np.count_nonzero(new != owner) > 0
            reset[shard.pairs_to_reset(owner, new, wl.grid)] = 1
            for x in sx:
                x.rebalance(new)
            owner = new
        _, own_b, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        keep = torch.from_numpy(owner[own_b]).cuda()
        for r in range(world):
            sx[r].send_phase({f: st[f][keep == r].contiguous() for f in FIELDS})
        outs = [x.outgoing() for x in sx]
        for r in range(world):
            sx[r].recv_phase({q: outs[q][r] for q in range(world) if q != r})
        for c in ctxs:
            c.status()
        # the single-rank oracle with the same raw pairs
        _, _, off, idx = oracle.pair_lists(g, own_b, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro = (None, None) if prev is None else prev[0]
        code, wire, wo, wlen, nxt = oracle.encode_all(rec, off, ra, ro, reset=reset)
        assert code == oracle.OK
        va, vo = (None, None) if prev is None else prev[1]
        code, recv, roff = oracle.decode_all(wire, wo, va, vo)
        assert code == oracle.OK
        for r in range(world):
            x = sx[r]
            lw = x.wire.cpu().numpy()
            lwo = x.wire_off.cpu().numpy().view(np.uint64)
            lwl = x.wire_len.cpu().numpy().view(np.uint64)
            sref, soff = x.sender_ref()
            sref, soff = sref.cpu().numpy(), soff.cpu().numpy().view(np.uint64)
            for p in np.nonzero(owner[np.arange(P) // 27] == r)[0]:
                assert int(lwl[p]) == int(wlen[p])
                a = int(lwo[p])
                assert lw[a:a + int(lwl[p])].tobytes() == \
                    wire[int(wo[p]):int(wo[p]) + int(wlen[p])].tobytes(), (t, r, p)
                assert (oracle.arena_pair(sref, soff, p).tobytes()
                        == oracle.arena_pair(nxt, off, p).tobytes()), (t, r, p)
            rrec, rof = x.receiver_ref()
            rrec, rof = rrec.cpu().numpy(), rof.cpu().numpy().view(np.uint64)
            for p in x.plan.mine:
                assert (oracle.arena_pair(rrec, rof, p).tobytes()
                        == oracle.arena_pair(recv, roff, p).tobytes()), (t, r, p)
        prev = ((nxt, off), (recv, roff))
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_migration_ranks_match_one_rank(world):
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import shard
    wl = Workload("t", 50000, (0.0,) * 3, (120.0, 120.0, 80.0), (4, 3, 2), 10.0, 2, seed=43)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    B = oracle.n_pairs(g) // 27
    s0, s1 = (to_numpy(x) for x in Generator(wl).series(2))
    _, own, _ = oracle.classify(g, s0["x"], s0["y"], s0["z"])
    perm = np.argsort(own, kind="stable")
    box_off = np.zeros(B + 1, dtype=np.uint64)
    box_off[1:] = np.cumsum(np.bincount(own, minlength=B))
    moved = {k: np.ascontiguousarray((s1 if k in ("x", "y", "z") else s0)[k][perm]) for k in s0}
    rng = np.random.default_rng(5)
    far = rng.choice(moved["x"].shape[0], 300, replace=False)
    for a, k in enumerate(("x", "y", "z")):
        moved[k][far] = rng.uniform(wl.lo[a], wl.hi[a], far.size)
    ref = oracle.migrate(g, moved, box_off)
    assert ref["status"] == oracle.OK
    owner = shard.slab_owners(B, world)
    cnt = np.diff(box_off.astype(np.int64))
    ctxs, mig, parts = [], [], []
    for r in range(world):
        mine = owner == r
        loff = np.zeros(B + 1, dtype=np.int64)
        loff[1:] = np.cumsum(np.where(mine, cnt, 0))
        sel = np.concatenate([np.arange(box_off[k], box_off[k + 1]) for k in np.nonzero(mine)[0]]
                             ).astype(np.int64)
        local = {k: torch.from_numpy(np.ascontiguousarray(
            moved[k][sel].view(np.int64) if k == "id" else moved[k][sel])).cuda() for k in FIELDS}
        ctxs.append(tera.Context(wl.lo, wl.hi, wl.grid, wl.w))
        mig.append(shard.ShardedMigration(ctxs[r], owner, r, world, 60000, 60000))
        parts.append(mig[r].send_phase(local, torch.from_numpy(loff).cuda()))
    outs = [m.outgoing() for m in mig]
    gb = ref["box_off_next"].astype(np.int64)
    for r in range(world):
        nxt, fin = mig[r].recv_phase(parts[r][0], parts[r][1],
                                     {q: outs[q][r] for q in range(world) if q != r})
        ctxs[r].status()
        fb = fin.cpu().numpy()
        for k in range(B):
            if owner[k] != r:
                assert fb[k + 1] == fb[k]
                continue
            a, b = int(gb[k]), int(gb[k + 1])
            c, d = int(fb[k]), int(fb[k + 1])
            assert b - a == d - c, k
            for f in FIELDS:
                got = nxt[f][c:d].cpu().numpy()
                want = ref["next"][f][a:b]
                assert got.tobytes() == want.tobytes(), (r, k, f)
    for c in ctxs:
        c.close()


def test_single_rank_sharded_exchange_is_the_plain_exchange():
    # one rank owning every box: nothing is routed, and the outputs are the oracle's
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import shard
    wl = Workload("t", 30000, (0.0,) * 3, (120.0, 120.0, 60.0), (3, 3, 2), 12.0, 3, seed=3)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    B = oracle.n_pairs(g) // 27
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    sx = shard.ShardedExchange(ctx, np.zeros(B, dtype=np.int32), 0, 1, 40000, 150000)
    ref = recv_ref = None
    for full in Generator(wl, device="cuda").series(3):
        st = {f: full[f] for f in FIELDS}
        sx.step(st, None)
        ctx.status()
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
        E = int(res["pair_off"][-1]) + oracle.n_pairs(g)
        sref, _ = sx.sender_ref()
        rrec, roff = sx.receiver_ref()
        assert sref[:E * 64].cpu().numpy().tobytes() == res["ref_next"][:E * 64].tobytes()
        assert rrec[:E * 64].cpu().numpy().tobytes() == res["recv"][:E * 64].tobytes()
        ref = (res["ref_next"], res["pair_off"])
        recv_ref = (res["recv"], res["recv_off"])
    ctx.close()

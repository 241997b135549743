"""Parity of agent migration (paper Sec. 2.1 "Agent Migration") with the
oracle, byte for byte: inbox offsets, the raw TAIO inbox arena, the next box
offsets and every column of the next box-major state, over chains of steps.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, Generator, Workload, scaled, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def to_dev(h):
    out = {}
    for k in FIELDS:
        a = np.ascontiguousarray(h[k])
        out[k] = torch.from_numpy(a.view(np.int64) if k == "id" else a).cuda()
    return out


def box_major_host(g, h):
    s, o, _ = oracle.classify(g, h["x"], h["y"], h["z"])
    assert s == oracle.OK
    perm = np.argsort(o, kind="stable")
    nb = int(g.n[0] * g.n[1] * g.n[2])
    off = np.zeros(nb + 1, dtype=np.uint64)
    off[1:] = np.cumsum(np.bincount(o, minlength=nb))
    return perm, off


def compare(mig, res, nxt, bo, n, Q):
    assert res["status"] == oracle.OK
    io = mig.inbox_off.cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(io, res["inbox_off"])
    L = int(io[-1])
    got = mig.arena[:(L + Q) * 64].cpu().numpy()
    assert got.tobytes() == res["arena"][:(L + Q) * 64].tobytes(), "inbox arena"
    np.testing.assert_array_equal(bo.cpu().numpy().view(np.uint64), res["box_off_next"])
    h = to_numpy(nxt)
    for k in FIELDS:
        a = h[k].view(np.uint64)
        b = np.ascontiguousarray(res["next"][k]).view(np.uint64)
        np.testing.assert_array_equal(a, b, err_msg=f"column {k}")
    return L


def chain(tera, wl, steps, p_far=0.0, sigma=None, max_leavers=None):
    """Move-only dynamics: state t+1 is state t moved, in the same order; both
    sides migrate the box-major state step by step."""
    wl = scaled(wl, wl.n0, p_grow=0.0, p_divide=0.0, p_die=0.0,
                step_sigma=sigma or wl.step_sigma)
    gen = Generator(wl, device="cuda")
    states = list(gen.series(steps + 1))
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w, wl.periodic)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, periodic=wl.periodic)
    n = int(states[0]["x"].shape[0])
    mig = tera.Migration(ctx, n, max_leavers=max_leavers or n)
    rng = np.random.default_rng(wl.seed)
    h0 = to_numpy(states[0])
    # move-only dynamics keep every agent at the index equal to its id
    assert np.array_equal(h0["id"], np.arange(n, dtype=np.uint64))
    perm, off = box_major_host(g, h0)
    cur = {k: h0[k][perm] for k in FIELDS}
    leavers = []
    for t in range(1, steps + 1):
        ht = to_numpy(states[t])
        moved = {k: (ht[k][perm] if k in ("x", "y", "z") else cur[k]) for k in FIELDS}
        if p_far:
            far = rng.random(n) < p_far
            for a, k in enumerate("xyz"):
                v = rng.uniform(wl.lo[a], wl.hi[a], n)
                moved[k] = np.where(far, np.minimum(v, math.nextafter(wl.hi[a], wl.lo[a])),
                                    moved[k])
        moved = {k: np.ascontiguousarray(v) for k, v in moved.items()}
        res = oracle.migrate(g, moved, off)
        dev = to_dev(moved)
        nxt, bo = mig.step(dev, torch.from_numpy(off.view(np.int64)).cuda())
        code, _ = ctx.status(raise_on_error=False)
        assert code == tera.OK
        leavers.append(compare(mig, res, nxt, bo, n, ctx.n_pairs))
        # the next step starts from the migrated state, with the positions
        # of state t+1 of the same agents (index = id)
        perm = res["next"]["id"].astype(np.int64)
        cur = res["next"]
        off = res["box_off_next"]
    ctx.close()
    return leavers


def test_uniform_chain(tera):
    L = chain(tera, scaled(WORKLOADS["uniform_1m"], 200_000), 3, sigma=8.0)
    assert all(x > 0 for x in L)


def test_blobs_chain_with_far_moves(tera):
    L = chain(tera, scaled(WORKLOADS["blobs_16m"], 300_000), 2, sigma=20.0, p_far=0.01)
    assert all(x > 0 for x in L)


def test_toroidal_chain(tera):
    chain(tera, scaled(WORKLOADS["torus_1m"], 150_000), 3, sigma=15.0, p_far=0.002)


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2048, 2049, 4097, 70001])
def test_ragged_sizes(tera, n):
    wl = Workload("t", n, (0.0,) * 3, (90.0, 60.0, 90.0), (3, 2, 3), 12.0, 3, p_move=0.6,
                  step_sigma=4.0, boundary="toroidal", wrap_axes=5, seed=500 + n)
    chain(tera, wl, 2, p_far=0.01)


def test_regroup_from_box_zero(tera):
    wl = scaled(WORKLOADS["uniform_1m"], 123_457)
    st = next(iter(Generator(wl, device="cuda").series(1)))
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    n = int(st["x"].shape[0])
    mig = tera.Migration(ctx, n, max_leavers=n)
    nxt, bo = mig.regroup(st)
    h = to_numpy(st)
    off = np.full(ctx.n_pairs // 27 + 1, n, dtype=np.uint64)
    off[0] = 0
    res = oracle.migrate(g, h, off)
    compare(mig, res, nxt, bo, n, ctx.n_pairs)
    perm, off_ref = box_major_host(g, h)
    np.testing.assert_array_equal(bo.cpu().numpy().view(np.uint64), off_ref)
    np.testing.assert_array_equal(to_numpy(nxt)["id"], h["id"][perm])
    ctx.close()


def test_every_agent_leaves(tera):
    # every agent shifts one box along x on a toroidal x axis
    lo, hi, grid = (0.0, 0.0, 0.0), (40.0, 20.0, 20.0), (4, 2, 2)
    g = oracle.make_grid(lo, hi, grid, 1.0, 1)
    rng = np.random.default_rng(9)
    n = 50_000
    h = {"id": rng.permutation(n).astype(np.uint64)}
    for a, k in enumerate("xyz"):
        h[k] = rng.uniform(lo[a], hi[a], n)
    for k in ("diameter", "volume", "adherence", "density"):
        h[k] = rng.uniform(1, 2, n)
    perm, off = box_major_host(g, h)
    h = {k: np.ascontiguousarray(v[perm]) for k, v in h.items()}
    h["x"] = np.ascontiguousarray(np.mod(h["x"] + 10.0, 40.0))
    res = oracle.migrate(g, h, off)
    assert int(res["inbox_off"][-1]) == n
    ctx = tera.Context(lo, hi, grid, 1.0, periodic=1)
    mig = tera.Migration(ctx, n, max_leavers=n)
    nxt, bo = mig.step(to_dev(h), torch.from_numpy(off.view(np.int64)).cuda())
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    compare(mig, res, nxt, bo, n, ctx.n_pairs)
    ctx.close()


def test_errors(tera):
    lo, hi, grid = (0.0, 0.0, 0.0), (30.0, 10.0, 10.0), (3, 1, 1)
    ctx = tera.Context(lo, hi, grid, 1.0)
    h = {"id": np.arange(5, dtype=np.uint64), "x": np.array([12.0, 3.0, 8.0, 15.0, 25.0]),
         "y": np.full(5, 5.0), "z": np.full(5, 5.0), "diameter": np.ones(5),
         "volume": np.ones(5), "adherence": np.ones(5), "density": np.ones(5)}
    off = torch.tensor([0, 2, 4, 5], dtype=torch.int64, device="cuda")
    # two leavers and 81 headers need 83 units
    mig = tera.Migration(ctx, 5, max_leavers=1)
    mig.step(to_dev(h), off)
    code, req = ctx.status(raise_on_error=False)
    assert code == tera.ECAPACITY and req == 83
    mig = tera.Migration(ctx, 5, max_leavers=2)
    nxt, bo = mig.step(to_dev(h), off)
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    g = oracle.make_grid(lo, hi, grid, 1.0)
    compare(mig, oracle.migrate(g, h, off.cpu().numpy().view(np.uint64)), nxt, bo, 5, 81)
    # box offsets that do not end at n
    mig.step(to_dev(h), torch.tensor([0, 2, 4, 6], dtype=torch.int64, device="cuda"))
    assert ctx.status(raise_on_error=False)[0] == tera.EINVAL
    # an agent outside the domain
    hb = dict(h, x=np.array([12.0, 3.0, 8.0, 30.0, 25.0]))
    mig.step(to_dev(hb), off)
    assert ctx.status(raise_on_error=False)[0] == tera.EDOMAIN
    # a damaged inbox header is refused by the receiver
    dev = to_dev(h)
    nxt = mig.empty_like(dev)
    bo = torch.empty_like(off)
    mig.send(dev, off, nxt, bo)
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    q = 1 * 27 + 12
    u = int(mig.inbox_off[q]) + q
    mig.arena[u * 64 + 16] ^= 1
    mig.recv(nxt, bo)
    assert ctx.status(raise_on_error=False)[0] == tera.ECORRUPT
    ctx.close()


def test_full_size_sampled_boxes(tera):
    """The 100M-agent workload as bench.py --migration runs it: regroup from
    box 0, then one migration step of the workload's moves.  For sampled boxes
    the oracle classifies the agents of the box and of its 26 neighbours and
    the box's next contents (stayers, then immigrants by arrival side and
    index) are compared record by record; the offsets and the ids of all 100M
    agents are checked as a whole."""
    import dataclasses
    wl = dataclasses.replace(WORKLOADS["uniform_100m"], p_grow=0.0, p_divide=0.0, p_die=0.0)
    it = Generator(wl, device="cuda").series(2)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    n = wl.n0
    mig = tera.Migration(ctx, n, max_leavers=n)
    cur, off = mig.regroup(next(it))
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    st = next(it)
    moved = {k: (st[k][cur["id"]] if k in ("x", "y", "z") else cur[k]) for k in FIELDS}
    del st
    nxt, bo = mig.step(moved, off)
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    # conservation: the same ids, each once
    assert torch.equal(torch.sort(nxt["id"]).values, torch.sort(moved["id"]).values)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    gx, gy, gz = wl.grid
    offp = off.cpu().numpy().view(np.uint64)
    offn = bo.cpu().numpy().view(np.uint64)

    def box_agents(s):
        a, b = int(offp[s]), int(offp[s + 1])
        return {k: moved[k][a:b].cpu().numpy() for k in FIELDS}, a

    owner_cache = {}

    def owners_of(s):
        if s not in owner_cache:
            h, _ = box_agents(s)
            st_, o, _ = oracle.classify(g, h["x"], h["y"], h["z"])
            assert st_ == oracle.OK
            owner_cache[s] = (h, o)
        return owner_cache[s]

    for d in (0, (gx * gy * gz) // 2 + gx // 2, gx * gy * gz - 1):
        cx, cy, cz = d % gx, (d // gx) % gy, d // (gx * gy)
        h, o = owners_of(d)
        parts = [{k: h[k][o == d] for k in FIELDS}]
        incoming = []
        for oz in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for ox in (-1, 0, 1):
                    sx, sy, sz = cx + ox, cy + oy, cz + oz
                    if (ox, oy, oz) == (0, 0, 0) or not (0 <= sx < gx and 0 <= sy < gy and
                                                          0 <= sz < gz):
                        continue
                    s = sx + gx * (sy + gy * sz)
                    incoming.append(((ox + 1) + 3 * (oy + 1) + 9 * (oz + 1), s))
        for side, s in sorted(incoming):
            hs, os_ = owners_of(s)
            parts.append({k: hs[k][os_ == d] for k in FIELDS})
        exp = {k: np.concatenate([p_[k] for p_ in parts]) for k in FIELDS}
        a, b = int(offn[d]), int(offn[d + 1])
        assert b - a == len(exp["x"])
        for k in FIELDS:
            got = nxt[k][a:b].cpu().numpy()
            np.testing.assert_array_equal(got.view(np.uint64), exp[k].view(np.uint64),
                                          err_msg=f"box {d} column {k}")
    # every box's next size: stayers + immigrants = previous size - leavers + arrivals
    io = mig.inbox_off.cpu().numpy().view(np.uint64)
    assert int(offn[-1]) == n and np.all(np.diff(offn.astype(np.int64)) >= 0)
    arrivals = np.diff(io.astype(np.int64))[:27 * gx * gy * gz].reshape(-1, 27).sum(1)
    assert int(arrivals.sum()) == int(io[-1])
    ctx.close()

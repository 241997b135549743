"""Parity of the CUDA path with the oracle, byte for byte, step by step.

Every output of every step (owner, mask, pair counts/offsets/lists, packed
arena, wire slab offsets, each wire message, new sender reference, receive
offsets and receive buffers) is compared with the oracle on the same seeded
inputs, over chains of iterations so the references chain as well.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, Generator, Workload, scaled, to_numpy

pytestmark = pytest.mark.gpu


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def u8(t, n):
    return t[:n].cpu().numpy()


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def compare_iteration(ctx, ex, st, res, P):
    n = int(st["x"].shape[0])
    assert res["status"] == oracle.OK
    np.testing.assert_array_equal(ex.part.owner[:n].cpu().numpy(), res["owner"])
    np.testing.assert_array_equal(u32(ex.part.mask[:n]), res["mask"])
    np.testing.assert_array_equal(u64(ex.part.pair_count), res["pair_count"])
    off = res["pair_off"]
    np.testing.assert_array_equal(u64(ex.pair_off[ex.last]), off)
    E = int(off[-1])
    np.testing.assert_array_equal(u32(ex.part.pair_idx[:E]), res["pair_idx"])
    units = E + P
    assert bytes(u8(ex.rec, units * 64)) == bytes(res["rec"][:units * 64]), "packed arena"
    wo = res["wire_off"]
    np.testing.assert_array_equal(u64(ex.wire_off), wo)
    wl = res["wire_len"]
    np.testing.assert_array_equal(u64(ex.wire_len), wl)
    wire = u8(ex.wire, int(wo[-1]))
    for p in range(P):
        a, b = int(wo[p]), int(wo[p]) + int(wl[p])
        assert bytes(wire[a:b]) == bytes(res["wire"][a:b]), f"wire message of pair {p}"
    sref, _ = ex.sender_ref()
    assert bytes(u8(sref, units * 64)) == bytes(res["ref_next"][:units * 64]), "sender reference"
    rrec, roff = ex.receiver_ref()
    np.testing.assert_array_equal(u64(roff), res["recv_off"])
    assert bytes(u8(rrec, units * 64)) == bytes(res["recv"][:units * 64]), "receive buffers"
    return E, int(wl.sum())


def run_chain(tera, wl, iters, per_subdomain=False, max_records=None, device="cuda",
              path=None, tune=None, id_columns=True):
    gen = Generator(wl, device=device)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w, periodic=wl.periodic)
    states = list(gen.series(iters))
    nmax = max(int(s["x"].shape[0]) for s in states)
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=max_records or 4 * nmax + 1024,
                           per_subdomain=per_subdomain, path=path, tune=tune,
                           id_columns=id_columns)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w, wl.periodic)
    ref = recv_ref = None
    stats = []
    for st in states:
        ex.step(st)
        code, _ = ctx.status(raise_on_error=False)
        assert code == tera.OK, f"device status {code}"
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
        stats.append(compare_iteration(ctx, ex, st, res, ctx.n_pairs))
        ref = (res["ref_next"], res["pair_off"])
        recv_ref = (res["recv"], res["recv_off"])
    ctx.close()
    return stats


def test_uniform_4k_all_iterations(tera):
    wl = WORKLOADS["uniform_4k"]
    stats = run_chain(tera, wl, wl.iterations)
    assert all(E > 0 for E, _ in stats)


def test_uniform_1m_one_launch_per_subdomain(tera):
    wl = WORKLOADS["uniform_1m"]
    stats = run_chain(tera, wl, 6, per_subdomain=True)
    E, sent = stats[-1]
    assert sent < 64 * E / 2  # the difference codec pays off


def test_uniform_1m_all_pairs_at_once(tera):
    run_chain(tera, WORKLOADS["uniform_1m"], 4)


def test_blobs_skewed_boxes(tera):
    # blob population (dense, uneven boxes) at 1/16 of the agents
    run_chain(tera, scaled(WORKLOADS["blobs_16m"], 1 << 20), 3)


def test_drift_persistent_motion(tera):
    run_chain(tera, scaled(WORKLOADS["drift_16m"], 1 << 19), 3)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 255, 2047, 2048, 2049, 4097, 70001])
def test_ragged_population_sizes(tera, n):
    wl = Workload("t", n, (0.0,) * 3, (90.0, 60.0, 60.0), (3, 2, 2), 12.0, 3,
                  p_divide=0.05, p_die=0.05, seed=100 + n)
    run_chain(tera, wl, 3)


@pytest.mark.parametrize("path", ["all_pairs", "batched"])
def test_toroidal_domain(tera, path):
    # every axis wraps: the boxes on the faces also exchange with the
    # opposite face (Sec. 2.5 toroidal space boundary)
    stats = run_chain(tera, scaled(WORKLOADS["torus_1m"], 1 << 18), 4, path=path)
    assert all(E > 0 for E, _ in stats)


@pytest.mark.parametrize("wrap_axes", [1, 4, 5])
@pytest.mark.parametrize("n", [0, 1, 2049, 70001])
def test_toroidal_some_axes(tera, wrap_axes, n):
    # axes 0 and 2 have 3 boxes and may wrap; axis 1 (2 boxes) stays closed
    wl = Workload("t", n, (0.0,) * 3, (90.0, 60.0, 90.0), (3, 2, 3), 12.0, 3,
                  p_divide=0.05, p_die=0.05, boundary="toroidal", wrap_axes=wrap_axes,
                  seed=300 + n + wrap_axes)
    run_chain(tera, wl, 3)
    run_chain(tera, wl, 3, path="batched")


@pytest.mark.parametrize("path", ["all_pairs", "batched"])
@pytest.mark.parametrize("K", [2, 3])
def test_reference_interval(tera, path, K):
    # the message of iteration 0 and of every K-th iteration after it is the
    # reference of the next K iterations, on both sides (the oracle is given
    # that older reference explicitly)
    wl = Workload("t", 30000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 8,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=21)
    states = list(Generator(wl, device="cuda").series(wl.iterations))
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=4 * nmax + 1024, path=path,
                           ref_interval=K)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    res_of = {}
    wire = []
    for t, st in enumerate(states):
        ex.step(st)
        ctx.status()
        if t == 0:
            ref = recv = None
        else:
            r = res_of[K * ((t - 1) // K)]
            ref, recv = (r["ref_next"], r["pair_off"]), (r["recv"], r["recv_off"])
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv)
        compare_iteration(ctx, ex, st, res, ctx.n_pairs)
        res_of[t] = res
        wire.append(int(res["wire_len"].sum()))
    ctx.close()
    # a stale reference costs bytes: iterations K..2K-1 all use iteration 0's message
    assert wire[K] >= wire[1] if K > 1 else True


def test_single_box_grid_has_no_messages(tera):
    wl = Workload("t", 5000, (0.0,) * 3, (50.0,) * 3, (1, 1, 1), 10.0, 2, seed=4)
    stats = run_chain(tera, wl, 2)
    assert stats[0][0] == 0


def test_narrow_boxes_two_sided_aura(tera):
    # box side 50 < 2w: agents near both faces of a box go both ways
    wl = Workload("t", 20000, (0.0,) * 3, (150.0, 100.0, 100.0), (3, 2, 2), 30.0, 3,
                  p_grow=0.1, p_divide=0.01, p_die=0.01, seed=8)
    run_chain(tera, wl, 3)


def edge_state(seed, n=6000):
    """Agents exactly on box edges and aura thresholds, plus ulp neighbours."""
    import math
    rng = np.random.default_rng(seed)
    lo, hi, grid, w = (-10.0, 0.0, 5.0), (50.0, 40.0, 35.0), (3, 2, 3), 7.5
    E = [[lo[a] + ((hi[a] - lo[a]) * k) / grid[a] for k in range(grid[a])] + [hi[a]]
         for a in range(3)]
    pts = np.zeros((n, 3))
    for a in range(3):
        c = rng.uniform(lo[a], hi[a], n)
        pick = rng.random(n)
        k = rng.integers(0, grid[a] + 1, n)
        cand = np.array(E[a])[k]
        c = np.where(pick < 0.2, cand, c)
        c = np.where((pick >= 0.2) & (pick < 0.35), cand + w, c)
        c = np.where((pick >= 0.35) & (pick < 0.5), cand - w, c)
        up = np.nextafter(c, np.inf)
        c = np.where((pick >= 0.5) & (pick < 0.6), up, c)
        c = np.clip(c, lo[a], math.nextafter(hi[a], lo[a]))
        pts[:, a] = c
    st = dict(id=np.arange(n, dtype=np.int64) * 7 + 3, x=pts[:, 0], y=pts[:, 1], z=pts[:, 2],
              diameter=rng.uniform(8, 12, n), volume=rng.uniform(0, 1, n),
              adherence=rng.uniform(0.3, 0.7, n), density=np.ones(n))
    return (lo, hi, grid, w), st


def test_edges_and_thresholds(tera):
    (lo, hi, grid, w), st = edge_state(1)
    ctx = tera.Context(lo, hi, grid, w)
    ex = tera.AuraExchange(ctx, max_agents=len(st["x"]), max_records=200000)
    g = oracle.make_grid(lo, hi, grid, w)
    ref = recv_ref = None
    rng = np.random.default_rng(2)
    for it in range(3):
        tst = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
        ex.step(tst)
        ctx.status()
        res = oracle.exchange_iteration(g, {k: (v.view(np.uint64) if k == "id" else v)
                                            for k, v in st.items()}, ref=ref, recv_ref=recv_ref)
        compare_iteration(ctx, ex, tst, res, ctx.n_pairs)
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
        # next iteration: drop some agents, nudge others by one ulp, shuffle order
        keep = rng.random(len(st["x"])) > 0.1
        st = {k: v[keep] for k, v in st.items()}
        perm = rng.permutation(len(st["x"]))
        st = {k: np.ascontiguousarray(v[perm]) for k, v in st.items()}
        st["x"] = np.where(rng.random(len(st["x"])) < 0.3, np.nextafter(st["x"], -np.inf),
                           st["x"]).clip(lo[0], None)
    ctx.close()


@pytest.mark.parametrize("lo,hi,grid,w", [
    ((-1.0e9, 0.0, 5.0), (1.0e9, 1.0, 35.0), (256, 3, 1), 0.1),
    ((1.0e-3, -7.0, 0.0), (1.0e-3 + 97.0 * 0.37, 89.0, 2.0), (97, 89, 2), 0.05),
    ((3.0e15, -1.0, -1.0), (3.0e15 + 256.0, 1.0, 1.0), (32, 2, 2), 0.5),
    ((-500.0, -3.0e-3, -7.5), (500.0, 3.0e-3, 2.5), (10, 6, 5), 1.0e-4),
])
def test_classification_many_boxes_wide_domains(tera, lo, hi, grid, w):
    # the box index starts from a float32 estimate and is fixed by exact key
    # comparisons: every owner and mask must equal the oracle's, including
    # points on edges, on aura thresholds, one ulp away, and a little beyond
    # the thresholds (a relative 2^-17 of the largest magnitude)
    import math
    rng = np.random.default_rng(sum(grid))
    n = 50000
    pts = np.zeros((n, 3))
    for a in range(3):
        E = np.array([lo[a] + ((hi[a] - lo[a]) * k) / grid[a] for k in range(grid[a])] + [hi[a]])
        c = rng.uniform(lo[a], hi[a], n)
        pick = rng.random(n)
        cand = E[rng.integers(0, grid[a] + 1, n)]
        c = np.where(pick < 0.2, cand, c)
        c = np.where((pick >= 0.2) & (pick < 0.3), cand + w, c)
        c = np.where((pick >= 0.3) & (pick < 0.4), cand - w, c)
        c = np.where((pick >= 0.4) & (pick < 0.5), np.nextafter(c, np.inf), c)
        c = np.where((pick >= 0.5) & (pick < 0.6), np.nextafter(c, -np.inf), c)
        # just beyond the aura thresholds, either side of a box
        margin = math.ldexp(max(abs(lo[a]), abs(hi[a])), -17)
        u = rng.uniform(0.0, 2.0, n) * margin
        c = np.where((pick >= 0.6) & (pick < 0.7), cand + w + u, c)
        c = np.where((pick >= 0.7) & (pick < 0.8), cand - w - u, c)
        pts[:, a] = np.clip(c, lo[a], math.nextafter(hi[a], lo[a]))
    ctx = tera.Context(lo, hi, grid, w)
    part = tera.PartitionBuffers.allocate(n, ctx.n_pairs, 7 * n, torch.device("cuda"))
    st = {"id": torch.arange(n, dtype=torch.int64, device="cuda"),
          "x": torch.from_numpy(pts[:, 0].copy()).cuda(), "y": torch.from_numpy(pts[:, 1].copy()).cuda(),
          "z": torch.from_numpy(pts[:, 2].copy()).cuda()}
    for f in ("diameter", "volume", "adherence", "density"):
        st[f] = torch.ones(n, dtype=torch.float64, device="cuda")
    ctx.partition(st, part)
    ctx.status()
    g = oracle.make_grid(lo, hi, grid, w)
    code, owner, mask = oracle.classify(g, pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy())
    assert code == oracle.OK
    np.testing.assert_array_equal(part.owner[:n].cpu().numpy(), owner)
    np.testing.assert_array_equal(u32(part.mask[:n]), mask)
    ctx.close()


def test_special_float_values_round_trip(tera):
    n = 4000
    rng = np.random.default_rng(3)
    lo, hi, grid, w = (0.0,) * 3, (40.0,) * 3, (2, 2, 2), 10.0
    specials = np.array([0x7FF8000000000001, 0xFFF0000000000000, 0x7FF0000000000000,
                         0x8000000000000000, 0x0000000000000001, 0x000FFFFFFFFFFFFF,
                         0x7FF7FFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    base = dict(id=rng.permutation(10**6)[:n].astype(np.int64),
                x=rng.uniform(0, 40, n), y=rng.uniform(0, 40, n), z=rng.uniform(0, 40, n))
    g = oracle.make_grid(lo, hi, grid, w)
    ctx = tera.Context(lo, hi, grid, w)
    ex = tera.AuraExchange(ctx, max_agents=n, max_records=10 * n)
    ref = recv_ref = None
    for it in range(3):
        st = dict(base)
        for f in ("diameter", "volume", "adherence", "density"):
            st[f] = specials[rng.integers(0, 8, n)].view(np.float64)
        tst = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}
        ex.step(tst)
        ctx.status()
        res = oracle.exchange_iteration(g, {k: (v.view(np.uint64) if k == "id" else v)
                                            for k, v in st.items()}, ref=ref, recv_ref=recv_ref)
        compare_iteration(ctx, ex, tst, res, ctx.n_pairs)
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ctx.close()


def test_determinism(tera):
    wl = scaled(WORKLOADS["uniform_1m"], 200_000)
    outs = []
    for _ in range(2):
        gen = Generator(wl, device="cuda")
        ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
        ex = tera.AuraExchange(ctx, max_agents=300_000, max_records=1_000_000)
        for st in gen.series(3):
            ex.step(st)
        torch.cuda.synchronize()
        wo, wl_ = u64(ex.wire_off), u64(ex.wire_len)
        wire = u8(ex.wire, int(wo[-1]))
        msgs = b"".join(wire[int(a):int(a) + int(b)].tobytes() for a, b in zip(wo[:-1], wl_))
        rrec, roff = ex.receiver_ref()
        outs.append((msgs, u8(rrec, 64 * (int(u64(roff)[-1]) + ctx.n_pairs)).tobytes()))
        ctx.close()
    assert outs[0] == outs[1]

"""The learned predictor on the GPU: its gradient against the float64 oracle,
the residual codec against the oracle byte for byte (records and histories of
both sides, per-call and batched paths), deterministic training, and the
bytes a trained network saves over plain XOR differences."""
import math

import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, Generator, Workload, scaled, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def drift(n=60000, iters=6, seed=31):
    return Workload("drift", n, (0.0,) * 3, (600.0, 600.0, 300.0), (3, 3, 2), 30.0, iters,
                    layout="blobs", n_blobs=6, p_move=1.0, persistent=True, seed=seed)


def velocity_network():
    from test_oracle_mlp import velocity_network as v
    return v()


def test_gradient_matches_oracle(tera):
    rng = np.random.default_rng(3)
    n = 700
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = rng.standard_normal((n, 3)).astype(np.float32)
    flag = (rng.random(n) < 0.8).astype(np.float32)
    samples = np.concatenate([X, Y, flag[:, None]], axis=1).astype(np.float32)
    p = (rng.standard_normal(4931) * 0.2).astype(np.float32)
    ctx = tera.Context((0, 0, 0), (10, 10, 10), (1, 1, 1), 1.0)
    grad = torch.zeros(4931, dtype=torch.float32, device="cuda")
    nv = ctx.mlp_grad(torch.from_numpy(samples).cuda(), torch.from_numpy(p).cuda(), grad)
    keep = flag != 0
    assert nv == int(keep.sum())
    _, g64 = oracle.mlp_loss_grad(p.astype(np.float64), X[keep].astype(np.float64),
                                  Y[keep].astype(np.float64))
    g = grad.cpu().numpy().astype(np.float64)
    for lo, hi in ((0, 512), (512, 576), (576, 4672), (4672, 4736), (4736, 4928), (4928, 4931)):
        scale = np.abs(g64[lo:hi]).max()
        assert np.abs(g[lo:hi] - g64[lo:hi]).max() <= 1e-4 * scale + 1e-7
    ctx.close()


@pytest.mark.parametrize("clip", [0.0, 0.05, 1e9])
def test_sgd_step_with_clipping_matches_oracle(tera, clip):
    # one training step over every valid sample (tera_mlp_train, steps = 1,
    # batch = all) against the float64 oracle: gradient, then the clipped step
    rng = np.random.default_rng(6)
    n = 900
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = (rng.standard_normal((n, 3)) * 2.0).astype(np.float32)
    flag = (rng.random(n) < 0.9).astype(np.float32)
    samples = np.concatenate([X, Y, flag[:, None]], axis=1).astype(np.float32)
    p0 = (rng.standard_normal(4931) * 0.2).astype(np.float32)
    ctx = tera.Context((0, 0, 0), (10, 10, 10), (1, 1, 1), 1.0)
    keep = flag != 0
    pt = torch.from_numpy(p0.copy()).cuda()
    lr = 0.05
    nv = ctx.mlp_train(torch.from_numpy(samples).cuda(), pt, 1, int(keep.sum()), lr, clip)
    assert nv == int(keep.sum())
    _, g64 = oracle.mlp_loss_grad(p0.astype(np.float64), X[keep].astype(np.float64),
                                  Y[keep].astype(np.float64))
    want = oracle.mlp_sgd_clip(p0.astype(np.float64), g64, lr, clip)
    got = pt.cpu().numpy().astype(np.float64)
    norm = np.linalg.norm(g64)
    c = clip / norm if 0.0 < clip < norm else 1.0
    if clip == 0.05:
        assert c < 0.5  # the limit is in force
    # float32 gradient (1e-4 of each layer's largest entry) and float32 rounding of the parameters
    tol = lr * c * 1e-3 * np.abs(g64).max() + 4e-7 * np.abs(p0).max()
    assert np.abs(got - want).max() <= tol
    ctx.close()


def run_pred_chain(tera, wl, params, path, tune=None):
    gen = Generator(wl, device="cuda")
    states = list(gen.series(wl.iterations))
    return run_pred_states(tera, states, wl.lo, wl.hi, wl.grid, wl.w, params, path, tune)


def check_samples(samples, rec, off, ref, wire, wo, wl_, lo, w):
    """The encoder's training samples of every slot of every XOR-mode message
    against the oracle: the features (the cell count among them, as
    ncount / 32) and targets of each matched slot with a full history, a zero
    flag everywhere else.  Returns the number of valid samples."""
    ra, ro, rh = ref
    P = len(off) - 1
    valid = 0
    for p in range(P):
        if not wl_[p] or int(wire[int(wo[p]) + 12]) != oracle.MODE_XOR:
            continue
        refp = oracle.arena_pair(ra, ro, p)
        if not len(refp):
            continue
        msg = oracle.arena_pair(rec, off, p)
        where = {int(i): k for k, i in enumerate(msg[:, 0])}
        cnt = oracle.cell_counts(refp, lo, w)
        for j in range(len(refp)):
            row = samples[12 * (int(ro[p]) + j):12 * (int(ro[p]) + j + 1)]
            h = rh[48 * (int(ro[p]) + j):48 * (int(ro[p]) + j + 1)]
            ok, f = oracle.features(refp[j], h, int(cnt[j]))
            m = where.get(int(refp[j, 0]))
            if m is None or not ok:
                assert row[11] == 0.0, (p, j)
                continue
            assert row[11] == 1.0, (p, j)
            assert row[:8].tobytes() == f.tobytes(), (p, j, row[:8], f, int(cnt[j]))
            tgt = (msg[m, 1:4].view(np.float64) - refp[j, 1:4].view(np.float64)).astype(np.float32)
            assert row[8:11].tobytes() == tgt.tobytes(), (p, j)
            valid += 1
    return valid


def run_pred_states(tera, states, lo, hi, grid, w, params, path, tune=None, samples=False):
    """The predictor path over `states` against the oracle: every message, both
    sides' references and histories byte for byte; with samples, the encoder's
    training samples too (check_samples).  Returns the message modes."""
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(lo, hi, grid, w)
    pt = torch.from_numpy(params).cuda()
    mr = 4 * nmax + 1024
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=mr, path=path,
                           params=pt, tune=tune)
    g = oracle.make_grid(lo, hi, grid, w)
    ref = recv = None
    modes = []
    n_valid = 0
    for st in states:
        if samples:
            ex.samples = torch.zeros(12 * mr, dtype=torch.float32, device="cuda")
        ex.step(st)
        ctx.status()
        s = to_numpy(st)
        _, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        _, cnt, off, idx = oracle.pair_lists(g, owner, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro, rh = (None, None, None) if ref is None else ref
        st_, wire, wo, wl_, nxt, hn = oracle.encode_all_pred(rec, off, ra, ro, rh, params, lo, w)
        assert st_ == oracle.OK
        va, vo, vh = (None, None, None) if recv is None else recv
        st_, rcv, rvo, rhn = oracle.decode_all_pred(wire, wo, va, vo, vh, params, lo, w)
        assert st_ == oracle.OK
        if samples and ref is not None:
            n_valid += check_samples(ex.samples.cpu().numpy(), rec, off, ref, wire, wo, wl_, lo, w)
        P = ctx.n_pairs
        E = int(off[-1])
        gwo = ex.wire_off.cpu().numpy().view(np.uint64)
        gwl = ex.wire_len.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(gwo, wo)
        np.testing.assert_array_equal(gwl, wl_)
        gwire = ex.wire[:int(wo[-1])].cpu().numpy()
        for p in range(P):
            a, b = int(wo[p]), int(wo[p] + wl_[p])
            assert gwire[a:b].tobytes() == wire[a:b].tobytes(), f"message of pair {p}"
            if wl_[p]:
                modes.append(int(wire[a + 12]))
        sref, _ = ex.sender_ref()
        assert sref[:(E + P) * 64].cpu().numpy().tobytes() == nxt[:(E + P) * 64].tobytes()
        assert ex.sender_hist()[:E * 48].cpu().numpy().tobytes() == hn.tobytes()
        rr, ro_ = ex.receiver_ref()
        assert rr[:(E + P) * 64].cpu().numpy().tobytes() == rcv[:(E + P) * 64].tobytes()
        assert ex.receiver_hist()[:E * 48].cpu().numpy().tobytes() == rhn.tobytes()
        ref, recv = (nxt, off, hn), (rcv, rvo, rhn)
    ctx.close()
    if samples:
        assert n_valid > 0
    return modes


def cell_edges(lo, hi, w):
    """The first binary64 value of each cell 1 .. n - 1 of one axis (cell(x) =
    floor((x - lo) / w)), found by stepping from lo + k w one ulp at a time."""
    n = math.floor((hi - lo) / w) + 1
    out = []
    for k in range(1, n):
        x = lo + k * w
        while math.floor((x - lo) / w) >= k:
            x = math.nextafter(x, -math.inf)
        while math.floor((x - lo) / w) < k:
            x = math.nextafter(x, math.inf)
        out.append(x)
    return np.array(out)


def boundary_states(lo, hi, w, near, n, iters, seed):
    """Agents (same ids every iteration) placed on cell edges of each axis or
    within two ulps of one, re-drawn every iteration: per axis, the edges
    within 4 w of the `near` coordinates (the box faces, so that many agents
    are in some aura), which gives dozens of agents per cell on both sides of
    every edge."""
    rng = np.random.default_rng(seed)
    edges = []
    for a in range(3):
        e = cell_edges(lo[a], hi[a], w)
        sel = np.zeros(len(e), dtype=bool)
        for c in near[a]:
            sel |= np.abs(e - c) <= 4 * w
        edges.append(e[sel])
    d = 8.0 + 4.0 * rng.random(n)
    states = []
    for _ in range(iters):
        pos = []
        for a in range(3):
            x = edges[a][rng.integers(0, len(edges[a]), n)]
            k = rng.integers(-2, 3, n)
            for s in (1, 2):
                x = np.where(k >= s, np.nextafter(x, np.inf), x)
                x = np.where(k <= -s, np.nextafter(x, -np.inf), x)
            pos.append(np.clip(x, lo[a], np.nextafter(hi[a], -np.inf)))
        st = dict(id=np.arange(n, dtype=np.int64), x=pos[0], y=pos[1], z=pos[2], diameter=d,
                  volume=(math.pi / 6.0) * d ** 3, adherence=np.full(n, 0.5),
                  density=np.ones(n))
        states.append({k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()})
    return states


@pytest.mark.parametrize("path", ["batched", "all_pairs"])
def test_cell_counts_on_binary64_cell_edges(tera, path):
    """Every reference record on a cell edge or within two ulps of one (the
    device finds cells by the context's threshold tables, the oracle by the
    binary64 formula): the training samples' cell counts and features, the
    messages and both sides' histories all equal the oracle's."""
    lo, hi, w = (-37.5, 12.25, 0.0), (41.3, 70.0, 33.0), 0.7
    grid = (2, 2, 1)
    near = [[lo[0] + (hi[0] - lo[0]) / 2], [lo[1] + (hi[1] - lo[1]) / 2], [5.0, 20.0]]
    states = boundary_states(lo, hi, w, near, 20000, 5, seed=12)
    run_pred_states(tera, states, lo, hi, grid, w, velocity_network(), path, samples=True)


@pytest.mark.parametrize("path", ["all_pairs", "batched", "per_subdomain"])
def test_residual_codec_matches_oracle_velocity_net(tera, path):
    modes = run_pred_chain(tera, drift(), velocity_network(), path)
    assert oracle.MODE_RESIDUAL in modes and oracle.MODE_XOR in modes


@pytest.mark.parametrize("tune", [(256, 4, 0, 2), (128, 4, 0, 5), (256, 2, 0, 0)])
def test_residual_codec_carried_by_teams(tera, tune):
    # the predictor path with its heavy pairs carried by teams of blocks
    # (forced sizes, and sized by load): same bytes and histories as the oracle
    wl = Workload("drift", 150000, (0.0,) * 3, (600.0, 600.0, 300.0), (2, 2, 2), 30.0, 5,
                  layout="blobs", n_blobs=3, p_move=1.0, persistent=True, seed=77)
    modes = run_pred_chain(tera, wl, velocity_network(), "batched", tune=tune)
    assert oracle.MODE_RESIDUAL in modes


def test_residual_codec_with_global_hash_pairs(tera):
    # shared-memory tables limited to 32 records: every larger pair below the
    # team threshold is matched in the global hash segments by one block
    modes = run_pred_chain(tera, drift(), velocity_network(), "batched", tune=(256, 4, 32, 0))
    assert oracle.MODE_RESIDUAL in modes


@pytest.mark.parametrize("path", ["all_pairs", "batched"])
def test_residual_codec_matches_oracle_random_net(tera, path):
    rng = np.random.default_rng(9)
    params = (rng.standard_normal(4931) * 0.05).astype(np.float32)
    run_pred_chain(tera, drift(n=30000, iters=5, seed=8), params, path)


def test_training_is_deterministic_and_saves_bytes(tera):
    from paper_2509_24063_gb300 import predictor
    wl = drift(n=200000, iters=14, seed=41)
    states = list(Generator(wl, device="cuda").series(wl.iterations))
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    samples = predictor.collect(ctx, states[:10], nmax, 4 * nmax + 1024, every=1)
    trained = []
    for _ in range(2):
        p = predictor.init_params(5)
        nv = predictor.train(ctx, samples, p, steps=2000, batch=8192, lr=0.02, clip=1.0)
        assert nv > 10000
        trained.append(p.cpu().numpy().copy())
    assert trained[0].tobytes() == trained[1].tobytes()  # fixed-order sums
    eval_states = list(Generator(drift(n=200000, iters=8, seed=42), device="cuda").series(8))
    bx, rx = predictor.wire_bytes(ctx, eval_states, nmax, 4 * nmax + 1024)
    bp, rp = predictor.wire_bytes(ctx, eval_states, nmax, 4 * nmax + 1024,
                                  params=torch.from_numpy(trained[0]).cuda())
    assert rx == rp
    # the gain is bounded by the motion noise at byte granularity: a word only
    # shrinks when the residual is 256x smaller than the XOR difference
    assert bp < 0.995 * bx, (bp / rx, bx / rx)
    ctx.close()

"""The learned predictor on the GPU: its gradient against the float64 oracle,
the residual codec against the oracle byte for byte (records and histories of
both sides, per-call and batched paths), deterministic training, and the
bytes a trained network saves over plain XOR differences."""
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
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    pt = torch.from_numpy(params).cuda()
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=4 * nmax + 1024, path=path,
                           params=pt, tune=tune)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv = None
    modes = []
    for st in states:
        ex.step(st)
        ctx.status()
        s = to_numpy(st)
        _, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        _, cnt, off, idx = oracle.pair_lists(g, owner, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro, rh = (None, None, None) if ref is None else ref
        st_, wire, wo, wl_, nxt, hn = oracle.encode_all_pred(rec, off, ra, ro, rh, params, wl.lo,
                                                             wl.w)
        assert st_ == oracle.OK
        va, vo, vh = (None, None, None) if recv is None else recv
        st_, rcv, rvo, rhn = oracle.decode_all_pred(wire, wo, va, vo, vh, params, wl.lo, wl.w)
        assert st_ == oracle.OK
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
    return modes


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

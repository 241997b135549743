"""Checkpoint and resume of an aura-exchange chain: a chain stopped after a
few iterations, saved to a file (AuraExchange.checkpoint), and resumed in a
fresh context and exchange (restore) produces, in every later iteration, the
bytes of the uninterrupted chain: wire messages, sender reference, receive
buffers (and, on the predictor path, both sides' histories); with K = 1 the
resumed chain's last iteration is compared with the oracle as well."""
import numpy as np
import pytest
import torch

import oracle
from synth import Generator, Workload, to_numpy

from test_gpu_parity import compare_iteration, u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def snapshot(ex):
    """Bytes of the iteration just run (host copies): every wire message (not
    the unwritten rest of each pair's slab), both references, and histories."""
    P = ex.P
    wo = u64(ex.wire_off)
    wl = u64(ex.wire_len)
    wire = ex.wire[:int(wo[-1])].cpu().numpy()
    msgs = b"".join(wire[int(wo[p]):int(wo[p]) + int(wl[p])].tobytes() for p in range(P))
    sref, soff = ex.sender_ref()
    rrec, roff = ex.receiver_ref()
    E, R = int(u64(soff)[-1]), int(u64(roff)[-1])
    out = [wo.tobytes(), wl.tobytes(), msgs,
           u64(soff).tobytes(), sref[:(E + P) * 64].cpu().numpy().tobytes(),
           u64(roff).tobytes(), rrec[:(R + P) * 64].cpu().numpy().tobytes()]
    if ex.predictor:
        out += [ex.sender_hist()[:E * 48].cpu().numpy().tobytes(),
                ex.receiver_hist()[:R * 48].cpu().numpy().tobytes()]
    return out


def run_resumed(tera, tmp_path, wl, iters, stop, **kw):
    states = list(Generator(wl, device="cuda").series(iters))
    nmax = max(int(s["x"].shape[0]) for s in states)

    def make():
        ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
        return ctx, tera.AuraExchange(ctx, nmax, 4 * nmax + 1024, **kw)

    ctx, ex = make()
    whole = []
    for st in states:
        ex.step(st)
        ctx.status()
        whole.append(snapshot(ex))
    ctx.close()
    del ex
    ctx, ex = make()
    for st in states[:stop]:
        ex.step(st)
    ctx.status()
    path = tmp_path / "exchange.ckpt"
    torch.save(ex.checkpoint(), path)
    ctx.close()
    del ex
    ctx, ex = make()
    ex.restore(torch.load(path))
    for t in range(stop, iters):
        ex.step(states[t])
        ctx.status()
        got = snapshot(ex)
        for k, (a, b) in enumerate(zip(got, whole[t])):
            assert a == b, f"iteration {t}, output {k}"
    return ctx, ex, states


@pytest.mark.parametrize("path,K", [("batched", 1), ("all_pairs", 3), ("per_subdomain", 2),
                                    ("batched", 4)])
def test_resumed_chain_gives_the_same_bytes(tera, tmp_path, path, K):
    wl = Workload("t", 40000, (0.0,) * 3, (200.0, 150.0, 150.0), (4, 3, 3), 15.0, 7,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=51)
    ctx, ex, states = run_resumed(tera, tmp_path, wl, 7, 4, path=path, ref_interval=K)
    if K == 1:
        # the resumed chain's last iteration against the oracle's own chain
        g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
        ref = recv_ref = None
        for st in states:
            res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
            ref = (res["ref_next"], res["pair_off"])
            recv_ref = (res["recv"], res["recv_off"])
        compare_iteration(ctx, ex, states[-1], res, ctx.n_pairs)
    ctx.close()


def test_resumed_predictor_chain_gives_the_same_bytes(tera, tmp_path):
    from test_oracle_mlp import velocity_network
    wl = Workload("drift", 40000, (0.0,) * 3, (600.0, 600.0, 300.0), (3, 3, 2), 30.0, 6,
                  layout="blobs", n_blobs=6, p_move=1.0, persistent=True, seed=31)
    params = torch.from_numpy(velocity_network()).cuda()
    ctx, ex, _ = run_resumed(tera, tmp_path, wl, 6, 3, path="batched", params=params)
    ctx.close()


def test_restore_refuses_another_configuration(tera):
    ctx = tera.Context((0.0,) * 3, (100.0,) * 3, (2, 2, 2), 10.0)
    gen = Generator(Workload("t", 5000, (0.0,) * 3, (100.0,) * 3, (2, 2, 2), 10.0, 2, seed=3),
                    device="cuda")
    st = next(iter(gen.series(1)))
    ex = tera.AuraExchange(ctx, 6000, 30000, path="all_pairs", ref_interval=1)
    ex.step(st)
    state = ex.checkpoint()
    other = tera.AuraExchange(ctx, 6000, 30000, path="all_pairs", ref_interval=2)
    with pytest.raises(ValueError):
        other.restore(state)
    small = tera.AuraExchange(ctx, 6000, 16, path="all_pairs", ref_interval=1)
    with pytest.raises(ValueError):
        small.restore(state)
    ctx2 = tera.Context((0.0,) * 3, (100.0,) * 3, (2, 2, 2), 12.0)
    with pytest.raises(ValueError):
        tera.AuraExchange(ctx2, 6000, 30000, path="all_pairs").restore(state)
    ctx2.close()
    ctx.close()

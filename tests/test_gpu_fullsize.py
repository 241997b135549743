"""Parity at the benchmark's full size and launch configuration: the
100M-agent uniform workload (8x8x8 boxes) through the batched path replayed
from a CUDA graph with an autotuned schedule, as the benchmark times it.
The oracle recomputes the partition of all 100M agents of the third
iteration (pair offsets compared in full) and, for a sample of pairs
(including the largest), chains the per-pair codec over the three
iterations and compares the wire message, the sender's new reference and
the receiver's buffer of the graph-replayed iteration byte for byte."""
import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, Generator, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


def test_full_size_sampled_pairs():
    import paper_2509_24063_gb300 as tera
    wl = WORKLOADS["uniform_100m"]
    from paper_2509_24063_gb300 import autotune
    states = [{f: s[f] for f in FIELDS} for s in Generator(wl, device="cuda").series(3)]
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, nmax, int(nmax * 0.35) + 4096, path="batched")
    ex.step(states[0])
    autotune.tune_batched(ex, states[1], use_cache=False)  # runs iteration 1 too
    ctx.status()
    g = ex.capture(states[2], 2)
    g.replay()
    ex.advance()
    torch.cuda.synchronize()
    ctx.status()
    og = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    host = []
    for s in states:
        h = to_numpy(s)
        st, owner, mask = oracle.classify(og, h["x"], h["y"], h["z"])
        assert st == oracle.OK
        st, cnt, off, idx = oracle.pair_lists(og, owner, mask)
        assert st == oracle.OK
        host.append((h, off, idx))
    off1 = host[2][1]
    np.testing.assert_array_equal(ex.pair_off[ex.last].cpu().numpy().view(np.uint64), off1)
    counts = off1[1:] - off1[:-1]
    rng = np.random.default_rng(17)
    nonempty = np.nonzero(counts)[0]
    sample = set(rng.choice(nonempty, 40, replace=False).tolist())
    sample.add(int(np.argmax(counts)))
    wo = ex.wire_off.cpu().numpy().view(np.uint64)
    wlen = ex.wire_len.cpu().numpy().view(np.uint64)
    sref, soff = ex.sender_ref()
    rrec, roff = ex.receiver_ref()
    roff = roff.cpu().numpy().view(np.uint64)
    soff = soff.cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(roff, off1)

    def pair_records(h, off, idx, p):
        sub = idx[int(off[p]):int(off[p + 1])]
        recs = np.zeros((len(sub), 8), dtype=np.uint64)
        for w, f in enumerate(FIELDS):
            col = h[f] if f == "id" else h[f].view(np.uint64)
            recs[:, w] = col[sub]
        return recs

    for p in sorted(sample):
        ref = np.zeros((0, 8), np.uint64)
        for h in host[:2]:
            st, _, ref = oracle.encode_pair(pair_records(*h, p), ref, pair=p)
            assert st == oracle.OK
        r1 = ref
        st, wire, nxt = oracle.encode_pair(pair_records(*host[2], p), r1, pair=p)
        assert st == oracle.OK
        assert int(wlen[p]) == len(wire)
        got = ex.wire[int(wo[p]):int(wo[p]) + len(wire)].cpu().numpy()
        assert got.tobytes() == wire.tobytes(), f"wire message of pair {p}"
        a = (int(soff[p]) + p + 1) * 64
        assert sref[a:a + 64 * len(nxt)].cpu().numpy().tobytes() == nxt.tobytes()
        st, out = oracle.decode_pair(wire, r1, pair=p)
        assert st == oracle.OK
        a = (int(roff[p]) + p + 1) * 64
        assert rrec[a:a + 64 * len(out)].cpu().numpy().tobytes() == out.tobytes()
    ctx.close()

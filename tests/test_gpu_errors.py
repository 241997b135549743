"""Error paths of the CUDA path: every error is latched in the device status
word and returned by tera_ctx_status; no kernel traps.  Malformed messages are
built on the host; decode statuses are compared with the oracle's on the very
same bytes."""
import struct

import numpy as np
import pytest
import torch

import oracle
from synth import Generator, Workload, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def small(seed=21, n=6000, iters=2):
    wl = Workload("t", n, (0.0,) * 3, (120.0, 120.0, 60.0), (2, 2, 1), 25.0, iters,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=seed)
    return wl, list(Generator(wl, device="cuda").series(iters))


def test_domain_error_latched_and_agent_excluded(tera):
    wl, states = small()
    st = {k: v.clone() for k, v in states[0].items()}
    st["x"][5] = float("nan")
    st["y"][17] = wl.hi[1]
    st["z"][33] = -1.0
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    part = tera.PartitionBuffers.allocate(st["x"].shape[0], ctx.n_pairs, 100000, "cuda")
    ctx.partition(st, part)
    code, _ = ctx.status(raise_on_error=False)
    assert code == tera.EDOMAIN
    s = to_numpy(st)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ost, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
    assert ost == oracle.EDOMAIN
    np.testing.assert_array_equal(part.owner.cpu().numpy(), owner)
    np.testing.assert_array_equal(part.mask.cpu().numpy().view(np.uint32), mask)
    _, cnt, off, idx = oracle.pair_lists(g, owner, mask)
    np.testing.assert_array_equal(u64(part.pair_off), off)
    ctx.close()


def test_partition_capacity(tera):
    wl, states = small()
    st = states[0]
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    part = tera.PartitionBuffers.allocate(st["x"].shape[0], ctx.n_pairs, 10, "cuda")
    ctx.partition(st, part)
    code, req = ctx.status(raise_on_error=False)
    s = to_numpy(st)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    _, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
    _, cnt, off, idx = oracle.pair_lists(g, owner, mask)
    assert code == tera.ECAPACITY and req == int(off[-1])
    assert not u64(part.pair_off).any()  # every pair left empty
    # the context recovers once the capacity is sufficient
    part = tera.PartitionBuffers.allocate(st["x"].shape[0], ctx.n_pairs, req, "cuda")
    ctx.partition(st, part)
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    np.testing.assert_array_equal(u64(part.pair_off), off)
    ctx.close()


def test_wire_capacity(tera):
    wl, states = small()
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=20000, max_records=100000)
    ex.wire = ex.wire[:1024]
    ex.step(states[0])
    code, req = ctx.status(raise_on_error=False)
    assert code == tera.ECAPACITY and req > 1024
    ctx.close()


def exchanged(tera):
    """Two iterations; returns ctx, exchange and the oracle's receiver reference."""
    wl, states = small(iters=2)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=20000, max_records=100000)
    for st in states:
        ex.step(st)
    ctx.status()
    return ctx, ex


def message_with_holes_and_news(ex, P):
    wo, wl = u64(ex.wire_off), u64(ex.wire_len)
    wire = ex.wire.cpu().numpy()
    best = None
    for p in range(P):
        h = wire[int(wo[p]):int(wo[p]) + 64]
        ns, nn, nh = (int(v) for v in h[16:40].view(np.uint64))
        if ns > 2 and nn > 0 and nh > 0:
            best = p
            break
    assert best is not None
    return best, wo, wl, wire


def put(buf, off, fmt, v):
    buf[off:off + struct.calcsize(fmt)] = np.frombuffer(struct.pack(fmt, v), dtype=np.uint8)


MUTATIONS = {
    "magic": lambda w, ns, nn: put(w, 0, "<I", 0x41524555),
    "version": lambda w, ns, nn: put(w, 4, "<H", 9),
    "class": lambda w, ns, nn: put(w, 8, "<I", 99),
    "pair": lambda w, ns, nn: put(w, 48, "<I", 0xFFFF),
    "mode": lambda w, ns, nn: put(w, 12, "<I", 5),
    "n_slots": lambda w, ns, nn: put(w, 16, "<Q", ns + 1),
    "n_holes": lambda w, ns, nn: put(w, 32, "<Q", 0),
    "payload": lambda w, ns, nn: put(w, 40, "<Q", 1 << 40),
    "msg_bytes": lambda w, ns, nn: put(w, 56, "<Q", 16),
    "nibble_9": lambda w, ns, nn: put(w, 64 + 4 * (ns + nn - 1), "<I", 0x91),
    "nibble_15_w3": lambda w, ns, nn: put(w, 64 + 4 * (ns + nn - 1), "<I", 0xF001),
    "hole_among_new": lambda w, ns, nn: put(w, 64 + 4 * (ns + nn - 1), "<I", 0xF),
    "match_with_id_delta": lambda w, ns, nn: put(w, 64, "<I", 0x3),
    "overrun": lambda w, ns, nn: put(w, 64 + 4 * (ns + nn - 1), "<I", 0x88888888),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_malformed_message_status_matches_oracle(tera, name):
    ctx, ex = exchanged(tera)
    P = ctx.n_pairs
    p, wo, wl, wire = message_with_holes_and_news(ex, P)
    h = wire[int(wo[p]):int(wo[p]) + 64]
    ns, nn = int(h[16:24].view(np.uint64)[0]), int(h[24:32].view(np.uint64)[0])
    bad = wire.copy()
    msg = bad[int(wo[p]):int(wo[p + 1])]
    MUTATIONS[name](msg, ns, nn)
    # the oracle's verdict on the same bytes, against the same receiver reference
    rprev, roff_prev = ex.receiver_ref()
    # the reference the message was encoded against is the previous receive buffer
    rref = ex.recv[(ex.t) % 2].cpu().numpy()
    roff = u64(ex.recv_off[(ex.t) % 2])
    ref_recs = oracle.arena_pair(rref, roff, p)
    ost, _ = oracle.decode_pair(msg, ref_recs, pair=p, out_cap=10**6)
    assert ost != oracle.OK
    ex.wire.copy_(torch.from_numpy(bad).cuda())
    recv = torch.empty_like(ex.recv[0])
    recv_off = torch.empty_like(ex.recv_off[0])
    ctx.delta_decode(ex.wire, ex.wire_off, ex.recv[ex.t % 2], ex.recv_off[ex.t % 2], recv,
                     recv_off, p, p + 1)
    code, _ = ctx.status(raise_on_error=False)
    assert code == ost, (name, code, ost)
    ctx.close()


def test_unpack_inplace_and_validate(tera):
    ctx, ex = exchanged(tera)
    rrec, roff = ex.receiver_ref()
    off = u64(roff)
    P = ctx.n_pairs
    p = int(np.argmax(off[1:] - off[:-1]))
    start = (int(off[p]) + p) * 64
    n = int(off[p + 1] - off[p])
    view, cnt = ctx.unpack_inplace(rrec, start, (n + 1) * 64)
    assert cnt == n and view == rrec.data_ptr() + start + 64
    ctx.unpack_validate(rrec, roff)
    assert ctx.status(raise_on_error=False)[0] == tera.OK
    with pytest.raises(tera.TeraError):
        ctx.unpack_inplace(rrec, start, n * 64)  # too short for the count
    bad = rrec.clone()
    bad[start + 8] ^= 1  # class id
    with pytest.raises(tera.TeraError):
        ctx.unpack_inplace(bad, start, (n + 1) * 64)
    ctx.unpack_validate(bad, roff)
    assert ctx.status(raise_on_error=False)[0] == tera.ECORRUPT
    ctx.close()


def test_reset_reference_sends_raw(tera):
    wl, states = small(iters=3)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=20000, max_records=100000)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv_ref = None
    for t, st in enumerate(states):
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
        reset = None
        if t == 2:
            off = res["pair_off"]
            p = int(np.argmax(off[1:] - off[:-1]))
            ctx.reset_reference(p)
            reset = np.zeros(ctx.n_pairs, np.uint8)
            reset[p] = 1
            ost, wire, wo, wlen, nxt = oracle.encode_all(res["rec"], off, *ref, reset=reset)
            assert ost == oracle.OK
        ex.step(st)
        ctx.status()
        if t == 2:
            assert int(u64(ex.wire_len)[p]) == int(wlen[p])
            a = int(wo[p])
            got = ex.wire[a:a + int(wlen[p])].cpu().numpy()
            assert got.tobytes() == wire[a:a + int(wlen[p])].tobytes()
            assert int(got[12:16].view(np.uint32)[0]) == oracle.MODE_RAW
            rrec, roff = ex.receiver_ref()
            units = int(off[-1]) + ctx.n_pairs
            assert rrec[:units * 64].cpu().numpy().tobytes() == nxt[:units * 64].tobytes()
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ctx.close()

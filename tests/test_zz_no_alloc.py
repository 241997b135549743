"""tera_delta_decode_noalloc: the decode step for callers that cannot allocate
device memory (a host whose device memory is all reserved by its own pool, a
loop that forbids allocation after start-up).  It uses one fixed scratch
array inside the library instead of a context's scratch.

Checked through the C ABI, on two consecutive calls per iteration:
  * its receive buffers and receive offsets equal, byte for byte, those of
    tera_delta_decode on the same messages and references;
  * on messages and references made by the oracle, they equal the oracle's
    own decode byte for byte (the codec is integer-exact: tolerance zero);
  * the documented limits: a receive buffer that is too small, more pairs than
    the fixed scratch holds, and a pair count that is not a multiple of 27.
This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import Generator, Workload, to_numpy

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _noalloc(lib, wire, wire_off, ref, ref_off, P, class_id, out, out_off, stream):
    req = C.c_uint64(7)
    code = lib.tera_delta_decode_noalloc(
        _p(wire), _p(wire_off), _p(ref), _p(ref_off), P, class_id, _p(out), out.numel() // 64,
        _p(out_off), C.byref(req), C.c_void_p(stream.cuda_stream))
    return code, req.value


WL = Workload("t", 20000, (0.0,) * 3, (150.0, 100.0, 100.0), (3, 2, 2), 20.0, 3,
              p_grow=0.1, p_divide=0.02, p_die=0.02, seed=77)


def test_noalloc_decode_equals_context_decode_on_consecutive_calls():
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    ctx = tera.Context(WL.lo, WL.hi, WL.grid, WL.w)
    ex = tera.AuraExchange(ctx, max_agents=40000, max_records=400000)
    P = ctx.n_pairs
    stream = torch.cuda.current_stream()
    calls = 0
    for t, st in enumerate(Generator(WL, device="cuda").series(3)):
        ex.step(st)
        ctx.status()
        # inputs the context decode just used, and its outputs
        first = t == 0
        ref = None if first else ex.recv[ex.t % 2]
        ref_off = None if first else ex.recv_off[ex.t % 2]
        want, want_off = ex.receiver_ref()
        used = (int(want_off[-1].item()) + P) * 64
        for _ in range(2):
            out = torch.full_like(ex.recv[0], 0xA5)
            out_off = torch.full_like(ex.recv_off[0], -1)
            code, req = _noalloc(lib, ex.wire, ex.wire_off, ref, ref_off, P, ctx.class_id, out,
                                 out_off, stream)
            assert code == tera.OK
            assert req == 0
            np.testing.assert_array_equal(out_off.cpu().numpy(), want_off.cpu().numpy())
            assert out[:used].cpu().numpy().tobytes() == want[:used].cpu().numpy().tobytes()
            calls += 1
    assert calls == 6
    # a capacity limit is reported, not exceeded
    small = torch.empty(64 * 4, dtype=torch.uint8, device="cuda")
    small_off = torch.empty_like(ex.recv_off[0])
    code, req = _noalloc(lib, ex.wire, ex.wire_off, ex.recv[ex.t % 2], ex.recv_off[ex.t % 2], P,
                         ctx.class_id, small, small_off, stream)
    assert code == tera.ECAPACITY and req > 4
    # argument limits, rejected before any launch
    code, req = _noalloc(lib, ex.wire, ex.wire_off, None, None, 27 * 1214, ctx.class_id, small,
                         small_off, stream)
    assert code == tera.ECAPACITY and req == 0
    code, _ = _noalloc(lib, ex.wire, ex.wire_off, None, None, 28, ctx.class_id, small, small_off,
                       stream)
    assert code == tera.EINVAL
    ctx.close()


def test_noalloc_decode_equals_oracle_decode(oracle):
    """Messages and references from the oracle's own iterations; the
    no-allocation decode must rebuild exactly the oracle's receive buffers."""
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    g = oracle.make_grid(WL.lo, WL.hi, WL.grid, WL.w)
    P = oracle.n_pairs(g)
    stream = torch.cuda.current_stream()
    prev = None  # ((sender reference, offsets), (receiver reference, offsets))
    for st in Generator(WL, device="cpu").series(3):
        res = oracle.exchange_iteration(g, to_numpy(st),
                                        ref=None if prev is None else prev[0],
                                        recv_ref=None if prev is None else prev[1])
        assert res["status"] == oracle.OK
        wire, wire_off = _dev(res["wire"]), _dev(res["wire_off"].view(np.int64))
        ref = None if prev is None else _dev(prev[1][0])
        ref_off = None if prev is None else _dev(prev[1][1].view(np.int64))
        used = (int(res["recv_off"][-1]) + P) * 64
        for _ in range(2):
            out = torch.full((used + 64 * 64,), 0x5A, dtype=torch.uint8, device="cuda")
            out_off = torch.full((P + 1,), -1, dtype=torch.int64, device="cuda")
            code, req = _noalloc(lib, wire, wire_off, ref, ref_off, P, 1, out, out_off, stream)
            assert code == tera.OK and req == 0
            np.testing.assert_array_equal(out_off.cpu().numpy().view(np.uint64), res["recv_off"])
            assert out[:used].cpu().numpy().tobytes() == res["recv"][:used].tobytes()
        prev = ((res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"]))

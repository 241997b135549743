"""tera_delta_decode_noalloc: the decode step for callers that cannot allocate
device memory (a stream being captured into a graph, a host whose device
memory is all reserved by its own pool, a loop that forbids allocation after
start-up).  It uses one fixed scratch array inside the library instead of a
context's scratch.

Checked through the C ABI: on consecutive calls its receive buffers and
receive offsets equal, byte for byte, those of tera_delta_decode on the same
messages and references (the codec is integer-exact, so the tolerance is
zero).  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import Generator, Workload

pytestmark = pytest.mark.gpu


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def test_noalloc_decode_equals_context_decode_on_consecutive_calls():
    import paper_2509_24063_gb300 as tera
    from paper_2509_24063_gb300 import _lib
    lib = _lib.load()
    wl = Workload("t", 20000, (0.0,) * 3, (150.0, 100.0, 100.0), (3, 2, 2), 20.0, 3,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=77)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=40000, max_records=400000)
    P = ctx.n_pairs
    stream = torch.cuda.current_stream()
    calls = 0
    for t, st in enumerate(Generator(wl, device="cuda").series(3)):
        ex.step(st)
        ctx.status()
        # inputs the context decode just used, and its outputs
        first = t == 0
        ref = None if first else ex.recv[ex.t % 2]
        ref_off = None if first else ex.recv_off[ex.t % 2]
        want, want_off = ex.receiver_ref()
        used = (int(want_off[-1].item()) + P) * 64
        for _ in range(2 if t == 1 else 1):
            out = torch.full_like(ex.recv[0], 0xA5)
            out_off = torch.full_like(ex.recv_off[0], -1)
            req = C.c_uint64(7)
            code = lib.tera_delta_decode_noalloc(
                _p(ex.wire), _p(ex.wire_off), _p(ref), _p(ref_off), P, ctx.class_id, _p(out),
                out.numel() // 64, _p(out_off), C.byref(req), C.c_void_p(stream.cuda_stream))
            assert code == tera.OK
            assert req.value == 0
            np.testing.assert_array_equal(out_off.cpu().numpy(), want_off.cpu().numpy())
            assert out[:used].cpu().numpy().tobytes() == want[:used].cpu().numpy().tobytes()
            calls += 1
    assert calls == 4
    # a capacity limit is reported, not exceeded
    small = torch.empty(64 * 4, dtype=torch.uint8, device="cuda")
    small_off = torch.empty_like(ex.recv_off[0])
    req = C.c_uint64(0)
    code = lib.tera_delta_decode_noalloc(
        _p(ex.wire), _p(ex.wire_off), _p(ex.recv[ex.t % 2]), _p(ex.recv_off[ex.t % 2]), P,
        ctx.class_id, _p(small), 4, _p(small_off), C.byref(req), C.c_void_p(stream.cuda_stream))
    assert code == tera.ECAPACITY and req.value > 4
    ctx.close()

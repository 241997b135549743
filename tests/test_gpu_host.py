"""Host-resident state: HostExchange steps (pinned inputs copied in, wire
messages written back into pinned host memory by tera_wire_to_host) give the
oracle's messages byte for byte; a host buffer that is too small latches
TERA_ECAPACITY with the length required."""
import numpy as np
import pytest
import torch

import oracle
from synth import Generator, Workload, to_numpy

pytestmark = pytest.mark.gpu

FIELDS = ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def workload(n=40000, iters=4, seed=77):
    return Workload("h", n, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, iters,
                    p_grow=0.1, p_divide=0.02, p_die=0.02, seed=seed)


def test_host_exchange_matches_oracle(tera):
    from paper_2509_24063_gb300.host import HostExchange
    wl = workload()
    states = [{f: s[f] for f in FIELDS} for s in Generator(wl, device="cpu").series(wl.iterations)]
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    hx = HostExchange(ctx, nmax, 4 * nmax + 1024, path="batched")
    outs = [torch.empty(hx.wire_capacity, dtype=torch.uint8).pin_memory() for _ in states]
    pend = [hx.step({f: s[f].pin_memory() for f in FIELDS}, out) for s, out in zip(states, outs)]
    counts = [p.wait() for p in pend]
    ctx.status()
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv = None
    for st, out, nb in zip(states, outs, counts):
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv)
        assert res["status"] == oracle.OK
        wo, wlen = res["wire_off"], res["wire_len"]
        assert nb == int(wo[-1])
        host = out.numpy()
        for p in range(ctx.n_pairs):
            a, b = int(wo[p]), int(wo[p]) + int(wlen[p])
            assert host[a:b].tobytes() == res["wire"][a:b].tobytes(), f"pair {p}"
        ref, recv = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ctx.close()


def test_wire_to_host_capacity(tera):
    wl = workload(n=20000, iters=1, seed=78)
    st = {f: v.cuda() for f, v in next(iter(Generator(wl, device="cpu").series(1))).items()
          if f in FIELDS}
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, 20000, 100000, path="batched")
    ex.step(st)
    ctx.status()
    small = torch.empty(1024, dtype=torch.uint8).pin_memory()
    count = torch.zeros(1, dtype=torch.int64).pin_memory()
    ctx.wire_to_host(ex.wire, ex.wire_off, small, count)
    torch.cuda.synchronize()
    code, req = ctx.status(raise_on_error=False)
    used = int(ex.wire_off[-1].item())
    assert code == tera.ECAPACITY and req == used and int(count[0]) == used
    with pytest.raises(TypeError):
        ctx.wire_to_host(ex.wire, ex.wire_off, small.cuda(), count)
    ctx.close()

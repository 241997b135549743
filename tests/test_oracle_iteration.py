"""Pins for the oracle's arena-level drivers over a chain of iterations
(paper Sec. 2.3: both sides of each pair hold the same reference and update it
every iteration).

Checked at every iteration of a small seeded series: the receiver's decoded
buffers equal the sender's new reference byte for byte; every decoded buffer
holds exactly the records of that pair's message (as a set); an unchanged
iteration sends nothing but headers and zero codes; and the whole-iteration
C driver equals the step-by-step drivers.
"""
import numpy as np
import pytest

from synth import Generator, Workload, to_numpy


def run_chain(oracle, wl, iters):
    gen = Generator(wl)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv_ref = None
    out = []
    for t, st_t in enumerate(gen.series(iters)):
        s = to_numpy(st_t)
        st, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        assert st == oracle.OK
        st, cnt, off, idx = oracle.pair_lists(g, owner, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro = (None, None) if ref is None else ref
        st, wire, wo, wl_, nxt = oracle.encode_all(rec, off, ra, ro)
        assert st == oracle.OK
        va, vo = (None, None) if recv_ref is None else recv_ref
        st, recv, rvo = oracle.decode_all(wire, wo, va, vo)
        assert st == oracle.OK
        np.testing.assert_array_equal(rvo, off)
        assert recv.tobytes() == nxt.tobytes()
        for p in range(wl.n_pairs):
            a = oracle.arena_pair(rec, off, p)
            b = oracle.arena_pair(recv, rvo, p)
            assert sorted(map(tuple, a.tolist())) == sorted(map(tuple, b.tolist()))
        out.append(dict(s=s, off=off, wire=wire, wo=wo, wl=wl_, nxt=nxt, recv=recv,
                        ref=ref, recv_ref=recv_ref))
        ref, recv_ref = (nxt, off), (recv, rvo)
    return g, out


def test_chain_small_uniform(oracle):
    wl = Workload("t", 3000, (0.0,) * 3, (120.0, 120.0, 60.0), (2, 2, 1), 20.0, 6,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=11)
    g, out = run_chain(oracle, wl, wl.iterations)
    raw = sum(int(o["off"][-1]) for o in out[1:]) * 64
    sent = sum(int(o["wl"].sum()) for o in out[1:])
    assert sent < raw  # the difference codec shrinks messages after iteration 0


def test_unchanged_iteration_sends_only_headers(oracle):
    wl = Workload("t", 2000, (0.0,) * 3, (90.0,) * 3, (3, 1, 1), 10.0, 2, p_move=0.0, seed=3)
    g, out = run_chain(oracle, wl, 2)
    o = out[1]
    P = wl.n_pairs
    for p in range(P):
        m = int(o["off"][p + 1] - o["off"][p])
        assert int(o["wl"][p]) == 64 + 4 * m + (-4 * m) % 16  # header + zero codes
        w = o["wire"][int(o["wo"][p]):int(o["wo"][p]) + int(o["wl"][p])]
        assert not w[64:].any()


def test_whole_iteration_driver_matches_steps(oracle):
    wl = Workload("t", 2500, (0.0,) * 3, (100.0, 100.0, 100.0), (2, 2, 2), 15.0, 3,
                  p_divide=0.05, p_die=0.05, seed=5)
    g, out = run_chain(oracle, wl, 3)
    o = out[2]
    res = oracle.exchange_iteration(g, o["s"], ref=o["ref"], recv_ref=o["recv_ref"])
    assert res["status"] == oracle.OK
    np.testing.assert_array_equal(res["pair_off"], o["off"])
    np.testing.assert_array_equal(res["wire_off"], o["wo"])
    np.testing.assert_array_equal(res["wire_len"], o["wl"])
    assert res["ref_next"].tobytes() == o["nxt"].tobytes()
    assert res["recv"][:o["recv"].size].tobytes() == o["recv"].tobytes()
    for p in range(wl.n_pairs):
        a, n = int(o["wo"][p]), int(o["wl"][p])
        assert res["wire"][a:a + n].tobytes() == o["wire"][a:a + n].tobytes()


def test_reset_pair_sends_raw(oracle):
    wl = Workload("t", 1500, (0.0,) * 3, (100.0, 100.0, 100.0), (2, 1, 1), 20.0, 2, seed=9)
    g, out = run_chain(oracle, wl, 2)
    o = out[1]
    P = wl.n_pairs
    reset = np.zeros(P, dtype=np.uint8)
    p = int(np.argmax(o["off"][1:] - o["off"][:-1]))
    reset[p] = 1
    rec = oracle.pack(o["s"], o["off"], np.concatenate(
        [oracle.pair_lists(g, *oracle.classify(g, o["s"]["x"], o["s"]["y"], o["s"]["z"])[1:])[3]]))
    st, wire, wo, wl_, nxt = oracle.encode_all(rec, o["off"], *o["ref"], reset=reset)
    assert st == oracle.OK
    h = wire[int(wo[p]):int(wo[p]) + 64]
    assert int(h[12:16].view(np.uint32)[0]) == oracle.MODE_RAW
    assert int(h[16:24].view(np.uint64)[0]) == 0
    st, recv, rvo = oracle.decode_all(wire, wo, *o["recv_ref"])
    assert st == oracle.OK
    assert recv.tobytes() == nxt.tobytes()


def test_chain_with_predictor_histories_stay_identical(oracle):
    """Residual mode over chained iterations: receiver records and histories
    equal the sender's every iteration, and the residual mode is used."""
    from test_oracle_mlp import velocity_network
    wl = Workload("t", 4000, (0.0,) * 3, (200.0, 200.0, 100.0), (2, 2, 1), 30.0, 6,
                  layout="blobs", n_blobs=3, p_move=1.0, persistent=True, seed=12)
    p = velocity_network()
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv = None
    modes = []
    for st_t in Generator(wl).series(wl.iterations):
        s = to_numpy(st_t)
        st, owner, mask = oracle.classify(g, s["x"], s["y"], s["z"])
        st, cnt, off, idx = oracle.pair_lists(g, owner, mask)
        rec = oracle.pack(s, off, idx)
        ra, ro, rh = (None, None, None) if ref is None else ref
        st, wire, wo, wl_, nxt, hn = oracle.encode_all_pred(rec, off, ra, ro, rh, p, wl.lo, wl.w)
        assert st == oracle.OK
        va, vo, vh = (None, None, None) if recv is None else recv
        st, rcv, rvo, rhn = oracle.decode_all_pred(wire, wo, va, vo, vh, p, wl.lo, wl.w)
        assert st == oracle.OK
        assert rcv.tobytes() == nxt.tobytes() and rhn.tobytes() == hn.tobytes()
        modes += [int(wire[int(wo[q]) + 12]) for q in range(wl.n_pairs) if wl_[q]]
        ref, recv = (nxt, off, hn), (rcv, rvo, rhn)
    assert oracle.MODE_RESIDUAL in modes


@pytest.mark.parametrize("threads", [2, 7])
def test_threaded_iteration_equals_single_threaded(oracle, threads):
    """The all-cores CPU baseline (agents and pairs spread over threads) gives
    the single-threaded iteration's outputs byte for byte, over a chain."""
    from synth import Generator, Workload, to_numpy
    wl = Workload("t", 30000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 3,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=9)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    prev = None
    for st in Generator(wl, device="cpu").series(3):
        soa = to_numpy(st)
        kw = {} if prev is None else dict(ref=prev[0], recv_ref=prev[1])
        a = oracle.exchange_iteration(g, soa, **kw)
        b = oracle.exchange_iteration(g, soa, threads=threads, **kw)
        assert a["status"] == b["status"] == oracle.OK
        for k in ("owner", "mask", "pair_count", "pair_off", "pair_idx", "rec", "wire",
                  "wire_off", "wire_len", "ref_next", "recv", "recv_off"):
            assert a[k].tobytes() == b[k].tobytes(), k
        prev = ((a["ref_next"], a["pair_off"]), (a["recv"], a["recv_off"]))

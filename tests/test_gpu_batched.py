"""The batched form: encode + decode of every pair in one persistent launch
(optionally replayed from CUDA graphs), checked byte for byte against the
oracle, and invariant under every schedule the autotuner can pick."""
import numpy as np
import pytest
import torch

import oracle
from synth import WORKLOADS, Generator, Workload, scaled, to_numpy

from test_gpu_parity import compare_iteration, run_chain, u64, u8

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tera():
    import paper_2509_24063_gb300 as t
    return t


def test_batched_uniform_4k_all_iterations(tera):
    wl = WORKLOADS["uniform_4k"]
    run_chain(tera, wl, wl.iterations, path="batched")


def test_batched_uniform_1m(tera):
    run_chain(tera, WORKLOADS["uniform_1m"], 4, path="batched")


def test_batched_skewed_blobs(tera):
    run_chain(tera, scaled(WORKLOADS["blobs_16m"], 1 << 20), 3, path="batched")


@pytest.mark.parametrize("tune", [None, (256, 4, 32, 0), (512, 2, 0, 0)])
def test_batched_without_id_columns(tera, tune):
    # ids read from the records themselves (tera_codec_batched): same bytes
    wl = Workload("t", 60000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 3,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=5)
    run_chain(tera, wl, 3, path="batched", tune=tune, id_columns=False)


def test_id_columns_hold_the_record_ids(tera):
    # tera_pack_ids' column is word 0 of every packed record, and the codec's
    # ref_next column is word 0 of every record of the new sender reference
    wl = Workload("t", 40000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 3,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=8)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=60000, max_records=200000, path="batched")
    P = ctx.n_pairs
    for st in Generator(wl, device="cuda").series(3):
        ex.step(st)
        ctx.status()
        off = u64(ex.pair_off[ex.last])
        E = int(off[-1])
        recs = ex.rec[:(E + P) * 64].cpu().numpy().view(np.uint64).reshape(-1, 8)
        sref = ex.ref[ex.last][:(E + P) * 64].cpu().numpy().view(np.uint64).reshape(-1, 8)
        units = np.concatenate([np.arange(int(off[p]) + p + 1, int(off[p + 1]) + p + 1)
                                for p in range(P)]).astype(np.int64)
        np.testing.assert_array_equal(u64(ex.rec_ids[:E]), recs[units, 0])
        np.testing.assert_array_equal(u64(ex.ref_ids[ex.last][:E]), sref[units, 0])
    ctx.close()


@pytest.mark.parametrize("n", [0, 1, 3, 2049, 70001])
def test_batched_ragged_sizes(tera, n):
    wl = Workload("t", n, (0.0,) * 3, (90.0, 60.0, 60.0), (3, 2, 2), 12.0, 3,
                  p_divide=0.05, p_die=0.05, seed=200 + n)
    run_chain(tera, wl, 3, path="batched")


@pytest.mark.parametrize("tune", [(128, 1, 0, 0), (128, 16, 32, 0), (256, 2, 0, 0),
                                  (256, 4, 1024, 0), (512, 1, 0, 0), (512, 2, 4096, 0),
                                  (1024, 1, 0, 0), (1024, 2, 64, 0)])
def test_batched_schedule_invariance(tera, tune):
    # every schedule gives the oracle's bytes (and so the same bytes as each
    # other); small table_records send most pairs to the global hash segments
    wl = Workload("t", 60000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 3,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=5)
    run_chain(tera, wl, 3, path="batched", tune=tune)


@pytest.mark.parametrize("tune", [None, (256, 4, 32, 0), (512, 2, 0, 0)])
def test_batched_skewed_pairs_carried_by_teams(tera, tune):
    # two dense blobs: a few pairs hold most records, so they exceed the
    # average load of a block and are carried by teams of blocks
    wl = Workload("t", 200000, (0.0,) * 3, (400.0, 400.0, 400.0), (2, 2, 2), 20.0, 3,
                  layout="blobs", n_blobs=2, p_grow=0.1, p_divide=0.02, p_die=0.02, seed=12)
    run_chain(tera, wl, 3, path="batched", tune=tune)


@pytest.mark.parametrize("tune", [(256, 4, 32, 2), (256, 2, 32, 3), (128, 4, 32, 7),
                                  (256, 1, 0, 32)])
def test_batched_forced_team_sizes(tera, tune):
    # every heavy pair carried by exactly team_blocks blocks: the bytes do not
    # depend on how a pair's tiles are split among the members
    wl = Workload("t", 200000, (0.0,) * 3, (400.0, 400.0, 400.0), (2, 2, 2), 20.0, 3,
                  layout="blobs", n_blobs=2, p_grow=0.1, p_divide=0.02, p_die=0.02, seed=12)
    run_chain(tera, wl, 3, path="batched", tune=tune)


def _two_face_pairs(n=100000):
    # 2 x 1 x 1 boxes: the two face pairs hold every record (about n/10 each)
    return Workload("t", n, (0.0,) * 3, (200.0, 100.0, 100.0), (2, 1, 1), 20.0, 2,
                    p_grow=0.1, p_divide=0.02, p_die=0.02, seed=31)


def test_team_wait_runs_out_and_latches_timeout(tera):
    # teams of 1024 blocks, but the launch has one block per SM: no team can
    # ever meet.  Each wait gives up after 50 us of the global timer, latches
    # TERA_ETIMEOUT and abandons its pair; the launch ends, and the context
    # stays usable (the next iteration with the default schedule is exact).
    import time
    wl = _two_face_pairs()
    states = list(Generator(wl, device="cuda").series(2))
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=150000, max_records=400000, path="batched",
                           tune=(256, 1, 32, 1024, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ex.step(states[0])
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    code, _ = ctx.status(raise_on_error=False)
    assert code == tera.ETIMEOUT
    assert elapsed < 5.0
    ex.tune = None
    ex.reset()
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv_ref = None
    for st in states:
        ex.step(st)
        ctx.status()
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
        compare_iteration(ctx, ex, st, res, ctx.n_pairs)
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ctx.close()


def test_team_members_meet_within_a_short_limit(tera):
    # the same pairs with teams that can meet (4 blocks each): a 20 ms limit
    # is never reached, and the bytes are the oracle's
    run_chain(tera, _two_face_pairs(), 2, path="batched", tune=(256, 1, 32, 4, 20000))


def test_graph_replay_matches_oracle(tera):
    wl = Workload("t", 50000, (0.0,) * 3, (200.0, 200.0, 100.0), (2, 2, 1), 20.0, 5,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=6)
    states = list(Generator(wl, device="cuda").series(5))
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=80000, max_records=400000, path="batched")
    ex.step(states[0])  # eager first iteration reserves all scratch
    ctx.status()
    graphs = [ex.capture(states[t], t) for t in range(1, 5)]
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    res = oracle.exchange_iteration(g, to_numpy(states[0]))
    ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    for t in range(1, 5):
        graphs[t - 1].replay()
        ex.advance()
        torch.cuda.synchronize()
        ctx.status()
        res = oracle.exchange_iteration(g, to_numpy(states[t]), ref=ref, recv_ref=recv_ref)
        compare_iteration(ctx, ex, states[t], res, ctx.n_pairs)
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ctx.close()


def test_batched_wire_capacity_reported(tera):
    wl = Workload("t", 6000, (0.0,) * 3, (120.0, 120.0, 60.0), (2, 2, 1), 25.0, 1, seed=21)
    st = next(Generator(wl, device="cuda").series(1))
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=20000, max_records=100000, path="batched")
    ex.wire = ex.wire[:1024]
    ex.step(st)
    code, req = ctx.status(raise_on_error=False)
    assert code == tera.ECAPACITY and req > 1024
    ctx.close()


def test_autotuner_picks_a_valid_schedule(tera, tmp_path, monkeypatch):
    from paper_2509_24063_gb300 import autotune
    monkeypatch.setenv("TERA_TUNE_CACHE", str(tmp_path / "tune.json"))
    wl = scaled(WORKLOADS["uniform_1m"], 300_000)
    states = list(Generator(wl, device="cuda").series(3))
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=400_000, max_records=1_500_000, path="batched")
    ex.step(states[0])
    tune, table = autotune.tune_batched(ex, states[1], use_cache=False)
    assert tune in autotune.CANDIDATES and len(table) >= 12
    assert autotune.load_cached(ctx, int(ex.pair_off[1][-1].item())) == tune
    # the tuned schedule continues the chain with the oracle's bytes
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv_ref = None
    for t in range(2):
        res = oracle.exchange_iteration(g, to_numpy(states[t]), ref=ref, recv_ref=recv_ref)
        ref, recv_ref = (res["ref_next"], res["pair_off"]), (res["recv"], res["recv_off"])
    ex.step(states[2])
    ctx.status()
    res = oracle.exchange_iteration(g, to_numpy(states[2]), ref=ref, recv_ref=recv_ref)
    compare_iteration(ctx, ex, states[2], res, ctx.n_pairs)
    ctx.close()


@pytest.mark.parametrize("order", ["shuffled", "few_swaps", "reversed"])
@pytest.mark.parametrize("id_columns", [True, False])
def test_batched_agent_orders(tera, order, id_columns):
    """Pairs whose id lists are both strictly ascending (agents in id order)
    are matched by a windowed search, the others by the hash index: a chain
    whose agents are re-ordered every iteration (all pairs unsorted, a few
    agents swapped so that some pairs are unsorted, and the order reversed)
    gives the oracle's bytes on every output, through both matches."""
    wl = Workload("t", 50000, (0.0,) * 3, (300.0, 200.0, 200.0), (3, 2, 2), 25.0, 4,
                  p_grow=0.1, p_divide=0.02, p_die=0.02, seed=17)
    rng = np.random.default_rng(23)
    states = []
    for st in Generator(wl, device="cuda").series(4):
        n = int(st["x"].shape[0])
        if order == "shuffled":
            perm = rng.permutation(n)
        elif order == "reversed":
            perm = np.arange(n)[::-1].copy()
        else:
            perm = np.arange(n)
            a = rng.choice(n, 40, replace=False)
            perm[a] = perm[np.roll(a, 1)]
        idx = torch.from_numpy(perm).cuda()
        states.append({f: st[f][idx].contiguous() for f in
                       ("id", "x", "y", "z", "diameter", "volume", "adherence", "density")})
    nmax = max(int(s["x"].shape[0]) for s in states)
    ctx = tera.Context(wl.lo, wl.hi, wl.grid, wl.w)
    ex = tera.AuraExchange(ctx, max_agents=nmax, max_records=4 * nmax + 1024, path="batched",
                           id_columns=id_columns)
    g = oracle.make_grid(wl.lo, wl.hi, wl.grid, wl.w)
    ref = recv_ref = None
    for st in states:
        ex.step(st)
        code, _ = ctx.status(raise_on_error=False)
        assert code == tera.OK, f"device status {code}"
        res = oracle.exchange_iteration(g, to_numpy(st), ref=ref, recv_ref=recv_ref)
        compare_iteration(ctx, ex, st, res, ctx.n_pairs)
        ref = (res["ref_next"], res["pair_off"])
        recv_ref = (res["recv"], res["recv_off"])
    ctx.close()

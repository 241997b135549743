"""Pins for the oracle of the learned predictor and the residual codec mode.

* training reference (float64): gradient against central finite differences;
* inference (float32, fixed fmaf order): against an exact-rational evaluation
  that rounds each fused multiply-add once to the nearest float32;
* zigzag hand vectors; history update and neighbour count hand cases;
* a hand-built network that outputs the last displacement: on constant
  velocity motion every position residual is zero, so the residual mode is
  chosen and its position codes are all zero;
* residual encode -> decode round trips (records and histories), and the XOR
  mode of the extended encoder equals the pinned plain encoder byte for byte.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest

IN, H, OUT = 8, 64, 3
OFF_W1, OFF_B1 = 0, 512
OFF_W2, OFF_B2 = 576, 576 + 4096
OFF_W3, OFF_B3 = 4736, 4736 + 192


def f32(x):
    return float(np.float32(x))


def f32_round(q: Fraction) -> float:
    """Nearest float32 (ties to even) of an exact rational."""
    if q == 0:
        return 0.0
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)
    quantum = Fraction(2) ** (e - 23)
    n = a / quantum
    fl = n.numerator // n.denominator
    rem = n - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    val = fl * quantum
    if val >= Fraction(2) ** 128:
        return s * float("inf")
    return s * float(val)


def fmaf_exact(a, b, c):
    return f32_round(Fraction(a) * Fraction(b) + Fraction(c))


def infer_exact(p, x):
    relu = lambda v: v if v > 0 else 0.0
    h1 = []
    for j in range(H):
        acc = float(p[OFF_B1 + j])
        for k in range(IN):
            acc = fmaf_exact(float(p[OFF_W1 + j * IN + k]), float(x[k]), acc)
        h1.append(relu(acc))
    h2 = []
    for j in range(H):
        acc = float(p[OFF_B2 + j])
        for k in range(H):
            acc = fmaf_exact(float(p[OFF_W2 + j * H + k]), h1[k], acc)
        h2.append(relu(acc))
    out = []
    for j in range(OUT):
        acc = float(p[OFF_B3 + j])
        for k in range(H):
            acc = fmaf_exact(float(p[OFF_W3 + j * H + k]), h2[k], acc)
        out.append(acc)
    return np.array(out, dtype=np.float32)


def test_parameter_count(oracle):
    assert oracle.NPARAM == 4931 == oracle.lib().or_mlp_nparam()


@pytest.mark.parametrize("seed", range(3))
def test_inference_equals_exact_fmaf_evaluation(oracle, seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(oracle.NPARAM) * 0.4).astype(np.float32)
    x = (rng.standard_normal(8) * 2).astype(np.float32)
    got = oracle.mlp_infer(p, x)
    want = infer_exact(p, x)
    assert got.view(np.uint32).tolist() == want.view(np.uint32).tolist()


def test_gradient_matches_central_differences(oracle):
    rng = np.random.default_rng(7)
    p = rng.standard_normal(oracle.NPARAM) * 0.3
    X = rng.standard_normal((6, 8))
    Y = rng.standard_normal((6, 3))
    loss, g = oracle.mlp_loss_grad(p, X, Y)
    idx = list(rng.choice(oracle.NPARAM, 80, replace=False)) + [OFF_B1, OFF_B2, OFF_B3,
                                                               OFF_W3 + 5, OFF_W1 + 3]
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp, _ = oracle.mlp_loss_grad(q, X, Y, with_grad=False)
        q[i] -= 2 * h
        lm, _ = oracle.mlp_loss_grad(q, X, Y, with_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    # loss is the mean over samples of the squared error summed over outputs
    o = np.array([[0.0] * 3] * 6)
    assert loss > 0


def test_sgd_step(oracle):
    import ctypes as C
    p = np.arange(oracle.NPARAM, dtype=np.float64)
    g = np.ones(oracle.NPARAM)
    oracle.lib().or_mlp_sgd_f64(p.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p), 0.5)
    assert np.array_equal(p, np.arange(oracle.NPARAM) - 0.5)


def test_sgd_step_with_global_norm_clipping(oracle):
    # a gradient of norm 5 (entries 3 and 4): clipped to norm 1 the step is
    # lr * (3, 4) / 5; unclipped (clip 0, or clip above the norm) it is lr * g
    p = np.linspace(-1.0, 1.0, oracle.NPARAM)
    g = np.zeros(oracle.NPARAM)
    g[7], g[4000] = 3.0, 4.0
    q = oracle.mlp_sgd_clip(p, g, 0.5, 1.0)
    d = p - q
    assert d[7] == pytest.approx(0.5 * 0.6, rel=1e-15) and d[4000] == pytest.approx(0.5 * 0.8, rel=1e-15)
    assert np.count_nonzero(d) == 2
    for clip in (0.0, -1.0, 5.0, 100.0):
        np.testing.assert_array_equal(oracle.mlp_sgd_clip(p, g, 0.5, clip), p - 0.5 * g)
    # any gradient above the limit: the step's norm is lr * clip, along -g
    rng = np.random.default_rng(4)
    g = rng.standard_normal(oracle.NPARAM) * 3.0
    q = oracle.mlp_sgd_clip(p, g, 0.25, 2.0)
    step = p - q
    assert np.linalg.norm(step) == pytest.approx(0.25 * 2.0, rel=1e-12)
    cos = step @ g / (np.linalg.norm(step) * np.linalg.norm(g))
    assert cos == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("d,z", [(0, 0), (-1, 1), (1, 2), (-2, 3), (2, 4),
                                 (2**63 - 1, 2**64 - 2), (-2**63, 2**64 - 1)])
def test_zigzag_vectors(oracle, d, z):
    assert oracle.zigzag(d) == z
    assert oracle.unzigzag(z) == d & (2**64 - 1)


def bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def rec(i, x, y, z, d=10.0):
    return np.array([i, bits(x), bits(y), bits(z), bits(d), bits(1.0), bits(0.5), bits(1.0)],
                    dtype=np.uint64)


def hist(xp, d2, n):
    h = np.zeros(48, dtype=np.uint8)
    h[0:24] = np.array([bits(v) for v in xp], dtype=np.uint64).view(np.uint8)
    h[24:36] = np.array(d2, dtype=np.float32).view(np.uint8)
    h[36:40] = np.array([n], dtype=np.uint32).view(np.uint8)
    return h


def test_history_update(oracle):
    r = rec(1, 10.5, 20.0, 30.25)
    h = hist((10.0, 19.0, 30.0), (0.1, 0.2, 0.3), 1)
    out = oracle.hist_next(r, h)
    assert [struct.unpack("<d", bytes(out[8 * a:8 * a + 8]))[0] for a in range(3)] == \
        [10.5, 20.0, 30.25]
    assert out[24:36].view(np.float32).tolist() == [f32(0.5), f32(1.0), f32(0.25)]
    assert int(out[36:40].view(np.uint32)[0]) == 2
    h2 = oracle.hist_next(r, hist((0, 0, 0), (0, 0, 0), 2))
    assert int(h2[36:40].view(np.uint32)[0]) == 2  # saturates at two steps
    h0 = oracle.hist_next(r, hist((9, 9, 9), (7, 7, 7), 0))
    assert int(h0[36:40].view(np.uint32)[0]) == 1 and not h0[24:36].any()
    assert not oracle.hist_next().any()  # a new record starts without history


def test_cell_counts_hand_case(oracle):
    lo, w = (0.0, 0.0, 0.0), 10.0
    refs = np.array([rec(0, 1, 1, 1), rec(1, 9.9, 5, 5), rec(2, 10, 5, 5), rec(3, 19, 1, 1),
                     rec(4, 5, 5, 10)])
    assert oracle.cell_counts(refs, lo, w).tolist() == [2, 2, 2, 2, 1]


def test_features(oracle):
    r = rec(1, 10.5, 20.0, 30.25, d=12.0)
    ok, f = oracle.features(r, hist((10.0, 19.0, 30.0), (0.1, -0.2, 0.3), 2), 5)
    assert ok == 1
    assert f.tolist() == [f32(0.5), f32(1.0), f32(0.25), f32(0.1), f32(-0.2), f32(0.3),
                          f32(1.2), f32(5 / 32)]
    ok, _ = oracle.features(r, hist((10.0, 19.0, 30.0), (0.1, 0.2, 0.3), 1), 5)
    assert ok == 0  # one step of history is not enough


def velocity_network():
    """Outputs the first three features (the last displacement) exactly."""
    p = np.zeros(4931, dtype=np.float32)
    for a in range(3):
        p[OFF_W1 + (2 * a) * IN + a] = 1.0       # h1[2a]   = relu(+f_a)
        p[OFF_W1 + (2 * a + 1) * IN + a] = -1.0  # h1[2a+1] = relu(-f_a)
        p[OFF_W2 + (2 * a) * H + 2 * a] = 1.0
        p[OFF_W2 + (2 * a + 1) * H + 2 * a + 1] = 1.0
        p[OFF_W3 + a * H + 2 * a] = 1.0
        p[OFF_W3 + a * H + 2 * a + 1] = -1.0
    return p


def test_constant_velocity_gives_zero_residuals(oracle):
    lo, w = (0.0, 0.0, 0.0), 25.0
    p = velocity_network()
    ref, hst, msg = [], [], []
    for i in range(20):
        x0, v = np.array([10.0 + i, 20.0, 30.0 + 2 * i]), np.array([0.5, -0.25, 0.125])
        ref.append(rec(i, *(x0 + 2 * v)))        # x_{t-1}
        hst.append(hist(x0 + v, v, 2))            # x_{t-2}, (float) displacement before it
        msg.append(rec(i, *(x0 + 3 * v)))         # x_t: same velocity
    ref, hst, msg = np.array(ref), np.stack(hst), np.array(msg)[::-1].copy()
    st, wire, nxt, hn = oracle.encode_pair_pred(msg, ref, hst, p, lo, w)
    assert st == oracle.OK
    assert int(wire[12:16].view(np.uint32)[0]) == oracle.MODE_RESIDUAL
    codes = wire[64:64 + 4 * 20].view(np.uint32)
    assert all(((int(c) >> 4) & 0xFFF) == 0 for c in codes)  # w1..w3: zero residuals
    st2, wire_x, nxt_x = oracle.encode_pair(msg, ref)
    assert len(wire) < len(wire_x)
    st, out, hout = oracle.decode_pair_pred(wire, ref, hst, p, lo, w)
    assert st == oracle.OK
    np.testing.assert_array_equal(out, nxt)
    np.testing.assert_array_equal(hout, hn)


def rand_case(rng, r, m, overlap=0.8):
    ids = rng.choice(10000, r + m, replace=False)
    ref_ids = ids[:r]
    keep = rng.random(r) < overlap
    msg_ids = np.concatenate([ref_ids[keep], ids[r:r + m - int(keep.sum())]]) \
        if m >= keep.sum() else ref_ids[keep][:m]
    rng.shuffle(msg_ids)
    pos = rng.uniform(0, 100, (r, 3))
    ref = np.array([rec(int(i), *pos[k]) for k, i in enumerate(ref_ids)]).reshape(-1, 8)
    hst = np.stack([hist(pos[k] - rng.normal(0, 0.5, 3), rng.normal(0, 0.5, 3),
                         int(rng.integers(0, 3))) for k in range(r)]) if r else \
        np.zeros((0, 48), np.uint8)
    where = {int(i): k for k, i in enumerate(ref_ids)}
    msg = []
    for i in msg_ids:
        if int(i) in where:
            x = pos[where[int(i)]] + rng.normal(0, 0.5, 3)
        else:
            x = rng.uniform(0, 100, 3)
        msg.append(rec(int(i), *x))
    return ref, hst, np.array(msg).reshape(-1, 8)


@pytest.mark.parametrize("seed", range(12))
def test_residual_round_trip(oracle, seed):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(4931) * 0.05).astype(np.float32)
    ref, hst, msg = rand_case(rng, int(rng.integers(0, 120)), int(rng.integers(0, 120)))
    for allow in (True, False):
        st, wire, nxt, hn = oracle.encode_pair_pred(msg, ref, hst, p, (0, 0, 0), 30.0,
                                                    allow_residual=allow)
        assert st == oracle.OK
        st, out, hout = oracle.decode_pair_pred(wire, ref, hst, p, (0, 0, 0), 30.0)
        assert st == oracle.OK
        np.testing.assert_array_equal(out, nxt)
        np.testing.assert_array_equal(hout, hn)
        if not allow:  # XOR mode: identical to the plain encoder
            st2, wire2, nxt2 = oracle.encode_pair(msg, ref)
            assert bytes(wire) == bytes(wire2)
            np.testing.assert_array_equal(nxt, nxt2)


def test_residual_needs_the_predictor_on_the_receiver(oracle):
    lo, w = (0.0, 0.0, 0.0), 25.0
    p = velocity_network()
    ref = np.array([rec(1, 11.0, 20.0, 30.0)])
    hst = np.stack([hist((10.5, 20.0, 30.0), (0.5, 0.0, 0.0), 2)])
    msg = np.array([rec(1, 11.5, 20.0, 30.0)])
    st, wire, nxt, hn = oracle.encode_pair_pred(msg, ref, hst, p, lo, w)
    assert int(wire[12:16].view(np.uint32)[0]) == oracle.MODE_RESIDUAL
    st, _, _ = oracle.decode_pair_pred(wire, ref, hst, None, lo, w)
    assert st == oracle.ECORRUPT

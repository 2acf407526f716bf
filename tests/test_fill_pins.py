"""Pins of the learned-fill oracle (oracle/learned_fill.py) against facts outside itself:
library routines for the special cases they cover (torch's bfloat16 conversion, scipy's
2-D correlation), hand-computed values, finite differences for the backward pass, the
main FP64 oracle's explicit per-pixel counters for the stale mask, exact affine data for
the target, and Adam's first steps worked out by hand."""
import numpy as np
import pytest
import torch

from oracle import learned_fill as lf

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_bf16_rounding_matches_torch_and_hand_cases():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-6, 6, size=20000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-30]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(lf.bf16(v), ref)
    # bfloat16 keeps 8 significant bits: ulp(1) = 2^-7; ties go to the even mantissa
    assert lf.bf16(1.0 + 2.0 ** -8) == 1.0
    assert lf.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert lf.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7


def test_conv_identity_shift_and_library():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7))
    W = np.zeros((1, 2, 3, 3))
    W[0, 0, 1, 1] = 1.0
    np.testing.assert_array_equal(lf.conv3x3(x, W, np.zeros(1))[0], x[0])
    # the top-left tap reads x[i-1, j-1]: the image moves down-right, zeros enter
    W = np.zeros((1, 2, 3, 3))
    W[0, 1, 0, 0] = 1.0
    out = lf.conv3x3(x, W, np.array([0.5]))[0]
    exp = np.full((5, 7), 0.5)
    exp[1:, 1:] += x[1, :-1, :-1]
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-15)
    # a general kernel: the sum over channels of scipy's 2-D correlation with zero fill
    from scipy.signal import correlate2d
    W = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    out = lf.conv3x3(x, W, b)
    for o in range(3):
        ref = b[o] + sum(correlate2d(x[c], W[o, c], mode="same", boundary="fill") for c in range(2))
        np.testing.assert_allclose(out[o], ref, rtol=0, atol=1e-12)


def test_conv_hand_example():
    x = np.arange(9, dtype=np.float64).reshape(1, 3, 3)   # [[0,1,2],[3,4,5],[6,7,8]]
    W = np.array([[1.0, 0.0, -1.0], [2.0, 0.0, -2.0], [1.0, 0.0, -1.0]]).reshape(1, 1, 3, 3)
    out = lf.conv3x3(x, W, np.zeros(1))[0]
    # centre: (0 - 2) + 2 (3 - 5) + (6 - 8) = -8; top-left corner: 0 + 2 (0 - 1) + (0 - 4) = -6
    assert out[1, 1] == -8.0
    assert out[0, 0] == -6.0
    assert out[2, 2] == 4 + 2 * 7 - 0  # (4 - 0) + 2 (7 - 0) + 0


def _tiny_problem(seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(size=lf.N_PARAMS) * 0.3
    xs = rng.normal(size=(2, 2, 6, 7))
    ts = rng.normal(size=(2, 6, 7))
    ms = rng.random((2, 6, 7)) < 0.6
    return theta, xs, ts, ms


def test_backward_matches_finite_differences():
    theta, xs, ts, ms = _tiny_problem(2)
    loss, g = lf.loss_and_grad(theta, xs, ts, ms, quantize=False)
    h = 1e-6
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(lf.N_PARAMS, 60, replace=False),
                          [lf.N_PARAMS - 1, 288, 288 + 16 + 2304]])  # b3, b1[0], b2[0]
    for i in idx:
        e = np.zeros(lf.N_PARAMS)
        e[i] = h
        lp, _ = lf.loss_and_grad(theta + e, xs, ts, ms, quantize=False)
        lm, _ = lf.loss_and_grad(theta - e, xs, ts, ms, quantize=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    # the loss itself: mean of squared masked residuals, by hand
    ys = [lf.forward(theta, x, quantize=False)["y"] for x in xs]
    ref = sum(float(((y - t)[m] ** 2).sum()) for y, t, m in zip(ys, ts, ms)) / ms.sum()
    assert abs(loss - ref) <= 1e-12 * max(1.0, ref)


def test_quantized_forward_rounds_weights_and_layer_inputs_only():
    theta, xs, _, _ = _tiny_problem(4)
    f = lf.forward(theta, xs[0])
    p = lf.unflatten(theta)
    np.testing.assert_array_equal(f["W2"], lf.bf16(p["W2"]))
    np.testing.assert_array_equal(f["xq"], lf.bf16(xs[0]))
    np.testing.assert_array_equal(f["a1q"], lf.bf16(np.maximum(f["z1"], 0)))
    np.testing.assert_array_equal(f["a2q"], lf.bf16(np.maximum(f["z2"], 0)))
    # with weights, b1, b2 already bfloat16 and x = 0: a1 = relu(b1) and a2 = relu(b2 + W2 * a1)
    # - take b2 = 0 and a single nonzero W2 tap of 1 so that a2 is a1 moved - are exact in
    # bfloat16; rounding then changes nothing, so the rounded and unrounded passes agree
    q = {k: (lf.bf16(v) if k in ("W1", "W3", "b1") else v) for k, v in p.items()}
    q["W2"] = np.zeros_like(p["W2"])
    q["W2"][:, :, 1, 1] = np.eye(16)
    q["b2"] = np.zeros(16)
    qt = lf.flatten(q)
    x = np.zeros_like(xs[0])
    np.testing.assert_array_equal(lf.forward(qt, x)["y"], lf.forward(qt, x, quantize=False)["y"])


def test_age_feature_and_stale_mask_by_hand():
    none = 0xFFFFFFFFFFFFFFFF
    last = np.array([99, 90, 80, 60, 0, none], dtype=np.uint64)
    age = lf.age_feature(100, 20, last)
    np.testing.assert_allclose(age, [1 / 20, 10 / 20, 1.0, 2.0, lf.A_MAX, lf.A_MAX])
    # window [h, k) = [80, 100): pixels whose last event precedes it are stale
    np.testing.assert_array_equal(lf.stale_mask(80, last), [False, False, False, True, True, False])
    # stale exactly when age > 1 (for pixels with events)
    has = last != np.uint64(none)
    np.testing.assert_array_equal(lf.stale_mask(80, last)[has], age[has] > 1.0)


def test_stale_mask_matches_the_event_oracle_counters(oracle_mod):
    import eventsim
    W, H = 16, 12
    ev = eventsim.random_events(W, H, 3000, seed=5)
    o = oracle_mod.Oracle(W, H, q_min=1, spatial_filter=1, blur_mode=1)
    o.push(ev)
    o.readout(int(ev[-1, 1]))
    st = o.state()
    explicit = (st["ever"] == 1) & (st["cnt"] == 0)
    np.testing.assert_array_equal(lf.stale_mask(st["h"], st["last"]), explicit)


def test_affine_target_exact_data():
    rng = np.random.default_rng(6)
    L = rng.normal(size=(8, 9))
    active = rng.random((8, 9)) < 0.5
    I = 3.0 * L + 2.0
    I[~active] += 5.0  # only the active pixels enter the fit
    T, a, b = lf.affine_target(L, I, active)
    assert abs(a - 3.0) < 1e-12 and abs(b - 2.0) < 1e-12
    np.testing.assert_allclose(T[active], L[active], atol=1e-12)
    np.testing.assert_allclose(T[~active], L[~active] + 5.0 / 3.0, atol=1e-12)
    # two points: the line through them
    T, a, b = lf.affine_target(np.array([0.0, 1.0]), np.array([1.0, 4.0]), np.array([True, True]))
    assert abs(a - 3.0) < 1e-15 and abs(b - 1.0) < 1e-15


def test_adam_first_steps_by_hand():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    t1, m, v = lf.adam_step(theta, m, v, g, 1, lr=0.01)
    # step 1: m_hat = g, v_hat = g^2, so the move is lr * g / (|g| + eps)
    np.testing.assert_allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    g2 = np.array([0.1, 1.0, 2.0])
    t2, m2, v2 = lf.adam_step(t1, m, v, g2, 2, lr=0.01)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(t2, t1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14, atol=1e-15)

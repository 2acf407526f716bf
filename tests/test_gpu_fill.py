"""The learned stale-pixel fill's CUDA kernels against the FP64 oracle
(oracle/learned_fill.py).

Tolerances come from the arithmetic.  Every layer takes BF16 inputs and accumulates in
FP32 on the tensor cores.  With inputs and weights on a coarse binary grid, conv1 is exact
in FP32, so both sides round a1 to BF16 identically; conv2 then differs by at most the FP32
accumulation bound dz2 = eps32 (2 n) (sum |W2| |a1| + |b2|), n = 145 terms, and a2 can round
to the neighbouring BF16 value only where it lies within dz2 of a rounding boundary; the
output differs by at most eps32 (2 n) (sum |W3| |a2| + |b3|) + conv(|W3|, dz2 + those
flips).  On arbitrary inputs a1 can also round differently on the two sides where it lies
within rounding noise of a tie; such pixels are bounded by the worst case of every a1 and
a2 flipping and must be rare.
"""
import numpy as np
import pytest
import torch

import eventsim
from oracle import learned_fill as lf

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
N_TERMS = 145


def _grid_theta(seed):
    """Weights and b1 on a 2^-8 grid (|w| < 1: exactly BF16), other biases arbitrary."""
    rng = np.random.default_rng(seed)
    p = {}
    for k in lf.ORDER:
        s = lf.SHAPES[k]
        if k in ("W1", "W2", "W3", "b1"):
            scale = {"W1": 120, "W2": 40, "W3": 40, "b1": 30}[k]
            p[k] = np.clip(np.round(rng.normal(size=s) * scale), -255, 255) / 256.0
        else:
            p[k] = rng.normal(size=s) * 0.1
    return lf.flatten(p)


def _grid_inputs(W, H, seed):
    """Inputs on a 2^-6 grid within [-4, 4]: at most 8 significant bits, exactly BF16."""
    rng = np.random.default_rng(seed)
    L = np.round(rng.normal(size=(H, W)) * 40) / 64.0
    L = np.clip(L, -4, 4)
    age = np.round(rng.uniform(0, 4, size=(H, W)) * 64) / 64.0
    stale = (rng.random((H, W)) < 0.5).astype(np.uint8)
    return np.stack([L, age]), stale


def _abs_conv(x, W):
    return lf.conv3x3(np.abs(x), np.abs(W), np.zeros(W.shape[0]))


def _bf16_ulp(v):
    """Spacing of the BF16 values at |v| (8 significant bits); 0 at 0."""
    a = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def _exact_path_bound(f, theta):
    """Bound for identical a1 roundings: FP32 accumulation of conv2 and conv3, and the
    a2 values it can move across a BF16 rounding boundary."""
    p = lf.unflatten(theta)
    dz2 = EPS32 * 2 * N_TERMS * (_abs_conv(f["a1q"], f["W2"]) + np.abs(p["b2"])[:, None, None])
    ulp2 = _bf16_ulp(f["a2q"])
    to_boundary = ulp2 / 2 - np.abs(f["a2"] - f["a2q"])
    flip2 = np.where(to_boundary <= dz2, np.maximum(ulp2, _bf16_ulp(f["a2"] + dz2)), 0.0)
    return (EPS32 * 2 * N_TERMS * (_abs_conv(f["a2q"], f["W3"])[0] + abs(p["b3"][0]))
            + _abs_conv(dz2 + flip2, f["W3"])[0])


def _flip_bound(f):
    """Worst case of every a1 and a2 value rounding to its BF16 neighbour."""
    da2 = _abs_conv(2.0 ** -7 * np.abs(f["a1q"]), f["W2"])
    return _abs_conv(da2 + 2.0 ** -7 * (np.abs(f["a2q"]) + da2), f["W3"])[0]


def _gpu_forward(theta, x, stale):
    from paper_2510_20071_gb300 import fill_forward
    xt = torch.from_numpy(x.astype(np.float32)).cuda().contiguous()
    st = torch.from_numpy(stale.astype(np.uint8)).cuda().contiguous()
    return fill_forward(theta.astype(np.float32), xt, st).cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("WH", [(1, 1), (7, 5), (126, 8), (127, 9), (300, 37), (1280, 24)])
def test_forward_exact_path_on_grid_inputs(WH):
    W, H = WH
    theta = _grid_theta(1)
    x, stale = _grid_inputs(W, H, 2)
    f = lf.forward(theta, x)
    ref = np.where(stale == 1, f["y"], x[0])
    got = _gpu_forward(theta, x, stale)
    bound = np.where(stale == 1, _exact_path_bound(f, theta), 0.0)
    err = np.abs(got - ref)
    assert np.all(err <= bound + 1e-30), (err.max(), bound[err > bound])
    # non-stale pixels are L exactly
    np.testing.assert_array_equal(got[stale == 0], x[0][stale == 0])


def test_forward_realistic_inputs_rare_rounding_flips():
    W, H = 333, 70
    from paper_2510_20071_gb300.fill import init_params
    theta = init_params(5).astype(np.float64)
    rng = np.random.default_rng(3)
    L = rng.normal(size=(H, W)) * 0.4
    age = np.minimum(4.0, rng.exponential(1.0, size=(H, W)))
    stale = (age > 1.0).astype(np.uint8)
    x = np.stack([L.astype(np.float32).astype(np.float64), age.astype(np.float32).astype(np.float64)])
    f = lf.forward(theta, x)
    ref = np.where(stale == 1, f["y"], x[0])
    got = _gpu_forward(theta, x, stale)
    err = np.abs(got - ref)[stale == 1]
    exact = _exact_path_bound(f, theta)[stale == 1]
    flips = _flip_bound(f)[stale == 1]
    assert np.all(err <= exact + flips)
    assert np.mean(err <= 4 * exact + 1e-7) >= 0.99, np.mean(err <= 4 * exact + 1e-7)


def _stream_handle_vs_oracles(oracle_mod, theta, W=96, H=72, n=60_000):
    from paper_2510_20071_gb300 import Fibar
    ev = eventsim.simulate(W, H, n, scene="perlin", seed=7, noise_frac=0.02)
    f = Fibar(W, H, c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=2)
    if theta is not None:
        f.set_fill_weights(theta.astype(np.float32))
    o = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=1)
    dev = ev.cuda()
    results = []
    for lo in range(0, n, 15_000):
        hi = lo + 15_000
        f.push(dev[lo:hi])
        o.push(ev[lo:hi])
        t = int(ev[hi - 1, 1])
        img = f.readout(t).cpu().numpy().astype(np.float64)
        s2 = o.readout(t)
        st = o.state()
        x_gpu, st_gpu = f.fill_features()
        results.append((img, s2, st, x_gpu.cpu().numpy(), st_gpu.cpu().numpy()))
    f.close()
    return results


def test_readout_with_learned_fill_matches_the_oracle_chain(oracle_mod):
    """blur_mode 2: the handle's image against the event oracle's state passed through the
    fill oracle; the handle's features against the oracle's L, age and stale mask."""
    from paper_2510_20071_gb300.fill import init_params
    theta = init_params(11).astype(np.float64)
    for img, _, st, xg, sg in _stream_handle_vs_oracles(oracle_mod, theta):
        H, W = img.shape
        L = st["L"].reshape(H, W)
        age = lf.age_feature(st["k"], st["q"], st["last"]).reshape(H, W)
        stale = lf.stale_mask(st["h"], st["last"]).reshape(H, W)
        np.testing.assert_array_equal(sg.astype(bool), stale)
        np.testing.assert_allclose(xg[0], L, atol=1e-4, rtol=0)
        np.testing.assert_allclose(xg[1], age, atol=0, rtol=2e-7)
        x = np.stack([L, age])
        f = lf.forward(theta, x)
        ref = np.where(stale, f["y"], L)
        err = np.abs(img - ref)
        # L itself differs from the oracle by up to 1e-4 (the filter's FP32 state), and its
        # BF16 rounding can differ by one BF16 step; through the network that moves y by at
        # most conv(|W3|, conv(|W2|, conv(|W1|, dL))) plus the later roundings' flips
        dl = np.stack([1e-4 + 2.0 ** -7 * np.abs(L), np.zeros_like(L)])
        p = lf.unflatten(theta)
        prop = _abs_conv(_abs_conv(_abs_conv(dl, f["W1"]), f["W2"]), f["W3"])[0]
        bound = np.where(stale, _exact_path_bound(f, theta) + _flip_bound(f) + prop, 1e-4)
        assert np.all(err <= bound), float((err - bound).max())
        assert np.mean(err[stale] <= 1e-3) >= 0.99


def test_learned_fill_without_weights_is_the_gaussian(oracle_mod):
    for img, s2, *_ in _stream_handle_vs_oracles(oracle_mod, None, n=30_000):
        assert np.abs(img - s2).max() <= 1e-4


def _train_problem(seed, W=64, H=48, F=3):
    rng = np.random.default_rng(seed)
    X = np.stack([_grid_inputs(W, H, seed * 10 + i)[0] for i in range(F)])
    T = rng.normal(size=(F, H, W)) * 0.5
    M = (rng.random((F, H, W)) < 0.5).astype(np.uint8)
    crops = np.array([[0, 0, 0], [1, 10, 17], [2, 24, 40], [0, 13, 5], [2, 0, 40], [1, 24, 2]], dtype=np.int32)
    return X, T, M, crops


def _oracle_batch(X, T, M, crops):
    S = 24
    xs = [X[f][:, y:y + S, x:x + S] for f, y, x in crops]
    ts = [T[f][y:y + S, x:x + S] for f, y, x in crops]
    ms = []
    for f, y, x in crops:
        m = M[f][y:y + S, x:x + S].astype(bool).copy()
        m[:3, :] = m[-3:, :] = False
        m[:, :3] = m[:, -3:] = False
        ms.append(m)
    return xs, ts, ms


def test_training_gradient_and_adam_step_match_the_oracle():
    from paper_2510_20071_gb300.fill import Frames, Trainer
    X, T, M, crops = _train_problem(3)
    theta0 = _grid_theta(4)
    fr = Frames(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(T.astype(np.float32)).cuda(),
                torch.from_numpy(M).cuda(), None)
    # a crop outside the frames is skipped and counted
    bad = np.array([[5, 0, 0], [0, 30, 0], [0, 0, 50]], dtype=np.int32)
    ct = torch.from_numpy(np.concatenate([crops, bad])).cuda()
    tr = Trainer(theta0.astype(np.float32))
    tr.step(fr, ct, lr=0.0)
    g_gpu = tr.grad.cpu().numpy().astype(np.float64)
    acc = tr.acc.cpu().numpy()
    assert acc[2] == 3.0
    xs, ts, ms = _oracle_batch(X, T.astype(np.float32).astype(np.float64), M, crops)
    loss, g = lf.loss_and_grad(theta0.astype(np.float32).astype(np.float64), xs, ts, ms)
    assert acc[1] == sum(int(m.sum()) for m in ms)
    assert abs(acc[0] / acc[1] - loss) <= 1e-5 * loss
    assert np.linalg.norm(g_gpu - g) <= 1e-4 * np.linalg.norm(g), np.linalg.norm(g_gpu - g) / np.linalg.norm(g)
    # one Adam step (step number 2 with the moments of step 1 = 0 here: a fresh trainer)
    tr2 = Trainer(theta0.astype(np.float32))
    lr = 1e-2
    tr2.step(fr, torch.from_numpy(crops).cuda(), lr=lr)
    th1 = tr2.params().astype(np.float64)
    ref1, _, _ = lf.adam_step(theta0.astype(np.float32).astype(np.float64), np.zeros(lf.N_PARAMS),
                              np.zeros(lf.N_PARAMS), g, 1, lr)
    sure = np.abs(g) > 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(th1[sure], ref1[sure], rtol=0, atol=1e-6)
    assert np.all(np.abs(th1 - theta0) <= lr * (1 + 1e-6) + 1e-7)

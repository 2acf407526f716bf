"""Host-side helpers of the learned fill (no GPU): the initial parameters and the affine
training target, the latter against the FP64 oracle's independent fit."""
import numpy as np
import torch

from oracle import learned_fill as lf


def test_init_params_layout_and_bounds():
    from paper_2510_20071_gb300 import FIBAR_FILL_NPARAMS
    from paper_2510_20071_gb300.fill import init_params
    th = init_params(3)
    assert th.dtype == np.float32 and th.size == FIBAR_FILL_NPARAMS == lf.N_PARAMS
    p = lf.unflatten(th)
    for k, cin in (("W1", 2), ("W2", 16)):
        lim = np.sqrt(6.0 / (9 * cin))
        assert np.abs(p[k]).max() <= lim + 1e-7 and np.abs(p[k]).max() > 0.5 * lim
    assert np.abs(p["W3"]).max() <= 0.1 * np.sqrt(6.0 / 144) + 1e-7
    for k in ("b1", "b2", "b3"):
        assert not p[k].any()
    np.testing.assert_array_equal(init_params(3), th)          # seeded
    assert not np.array_equal(init_params(4), th)


def test_affine_target_matches_the_oracle_fit():
    from paper_2510_20071_gb300.fill import affine_target
    rng = np.random.default_rng(9)
    L = rng.normal(size=(30, 40))
    I = 2.5 * L - 0.7 + rng.normal(scale=0.05, size=L.shape)
    active = rng.random(L.shape) < 0.4
    got = affine_target(torch.from_numpy(L).float(), torch.from_numpy(I).float(), torch.from_numpy(active))
    # the oracle fits the same float32 inputs in FP64
    ref, a, b = lf.affine_target(L.astype(np.float32), I.astype(np.float32), active)
    np.testing.assert_allclose(got.numpy(), ref, rtol=0, atol=2e-6)
    assert abs(a - 2.5) < 0.02 and abs(b + 0.7) < 0.02

"""Pins of the oracle's threshold calibration and correction (CPU only).

- relative thresholds (the paper's appendix on relative contrast thresholds): a
  hand-worked example (tests/golden), the identities the definitions imply (C' is the
  harmonic mean of C'_on and C'_off; the harmonic mean of C' over the sensor is 1), and
  recovery of known per-pixel thresholds from a simulated stationary recording;
- the Sec. 5.2 correction (Eq. 6's right-hand side times a per-pixel gain): a gain of 1
  changes nothing, a uniform gain scales every output (the filter and the blurs are
  linear, the detector does not read L), per-pixel gains scale each pixel without the
  spatial filter, and the first event from rest gives the closed form.
"""
import os

import numpy as np
import pytest
import torch

import eventsim
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "relative_thresholds_3x1.txt")


def _golden():
    evs, exp = [], {}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "events":
            evs.append((int(f[1]), int(f[2])))
        elif f[0] == "expect":
            exp[int(f[1])] = [float(v) for v in f[2:5]]
    x = torch.tensor([e[0] for e in evs])
    p = torch.tensor([e[1] for e in evs])
    ev = eventsim.pack_events(x, torch.zeros_like(x), p, torch.arange(len(evs)))
    return ev, exp


def test_relative_thresholds_hand_example():
    ev, exp = _golden()
    c_on, c_off, c = oracle.relative_thresholds(3, 1, ev)
    for i, (a, b, cc) in exp.items():
        np.testing.assert_allclose([c_on[0, i], c_off[0, i], c[0, i]], [a, b, cc], rtol=1e-15, equal_nan=True)


def test_relative_threshold_identities():
    ev = eventsim.random_events(17, 11, 20_000, seed=9, p_on=0.6)
    c_on, c_off, c = oracle.relative_thresholds(17, 11, ev)
    assert np.all(np.isfinite(c))  # every pixel has events of both signs here
    np.testing.assert_allclose(c, 2 * c_on * c_off / (c_on + c_off), rtol=1e-13)
    np.testing.assert_allclose(np.mean(1.0 / c), 1.0, rtol=1e-13)


def test_relative_thresholds_recover_simulated_sensor():
    """Known per-pixel ON/OFF thresholds watching a uniform triangle wave: the recovered
    relative thresholds equal C_on,i / C, C_off,i / C and C_i / C up to the pixels'
    hysteresis at the turning points (at most (C_on + C_off) of the amplitude per half
    period) and the count quantisation."""
    A = 20.0
    r = eventsim.threshold_recording(32, 24, periods=10, amplitude=A, steps_per_half=400)
    c_on, c_off, c = oracle.relative_thresholds(32, 24, r["events"])
    Ci = 2 * r["c_on"] * r["c_off"] / (r["c_on"] + r["c_off"])
    C = 1.0 / np.mean(1.0 / Ci)
    bound = 2 * np.max(r["c_on"] + r["c_off"]) / A
    for got, true in [(c_on, r["c_on"] / C), (c_off, r["c_off"] / C), (c, Ci / C)]:
        assert np.max(np.abs(got / true - 1)) < bound
    # a mistake in the formulas (a factor 2, ON and OFF swapped) is far outside the bound
    assert np.max(np.abs(c_off / (r["c_on"] / C) - 1)) > 2 * bound


def test_zero_counts_are_nan_and_outside_records_skipped():
    x = torch.tensor([0, 0, 5])
    ev = eventsim.pack_events(x, torch.zeros_like(x), torch.tensor([1, 1, 1]), torch.arange(3))
    c_on, c_off, c = oracle.relative_thresholds(2, 1, ev)
    assert c_on[0, 0] == 0.25 and np.isnan(c_off[0, 0]) and c[0, 0] == 0.5  # Nbar = 2 / 2 pixels
    assert np.isnan(c_on[0, 1]) and np.isnan(c_off[0, 1]) and np.isnan(c[0, 1])


def _run(W, H, ev, gain, t_reads, **params):
    o = oracle.Oracle(W, H, **params)
    if gain is not None:
        o.set_gain(gain)
    o.push(ev)
    imgs = [o.readout(t) for t in t_reads]
    st = o.state()
    o.close()
    return imgs, st


MODES = [dict(spatial_filter=0), dict(spatial_filter=1, blur_mode=0), dict(spatial_filter=1, blur_mode=1)]


@pytest.mark.parametrize("mode", MODES)
def test_gain_one_and_uniform_gain(mode):
    W, H = 24, 16
    ev = eventsim.random_events(W, H, 6000, seed=4)
    t = [1999, 3999, 5999]
    base, st0 = _run(W, H, ev, None, t, q_min=8, **mode)
    ones, st1 = _run(W, H, ev, np.ones(W * H), t, q_min=8, **mode)
    for a, b in zip(base, ones):
        np.testing.assert_array_equal(a, b)
    g = 1.7
    scaled, st2 = _run(W, H, ev, np.full(W * H, g), t, q_min=8, **mode)
    for a, b in zip(base, scaled):
        np.testing.assert_allclose(b, g * a, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(st0["cnt"], st2["cnt"])  # the detector ignores L
    np.testing.assert_array_equal(st0["pbar"], st2["pbar"])  # Eq. 7 is not scaled


def test_per_pixel_gain_without_spatial_filter():
    W, H = 20, 10
    ev = eventsim.random_events(W, H, 5000, seed=6)
    rng = np.random.default_rng(1)
    g = rng.uniform(0.5, 2.0, W * H)
    base, _ = _run(W, H, ev, None, [4999], spatial_filter=0)
    got, _ = _run(W, H, ev, g, [4999], spatial_filter=0)
    np.testing.assert_allclose(got[0].ravel(), g * base[0].ravel(), rtol=1e-12, atol=1e-13)


def test_gain_first_event_closed_form():
    """One ON event on a pixel at rest: p_bar = (1 - alpha) C_on, Eq. 6 gives
    C_on - p_bar = alpha C_on, times the gain G; L = (1 + beta) / 2 * G * alpha * C_on."""
    a, b = oracle.coefficients(40.0)
    G = 0.37
    ev = eventsim.pack_events(torch.tensor([1]), torch.tensor([0]), torch.tensor([1]), torch.tensor([0]))
    gain = np.ones(4)
    gain[1] = G
    imgs, st = _run(4, 1, ev, gain, [0], spatial_filter=0, c_on=0.25)  # exact in float32
    np.testing.assert_allclose(st["L"][1], 0.5 * (1 + b) * G * a * 0.25, rtol=1e-14)

"""The temporal filter's two schedules against the FP64 oracle, and the scan's speed.

The walk runs each 2x2 tile's events in arrival order in one thread; the scan composes
the per-event affine maps of Eqs. 7, 6, 10 along each pixel's events with a block-wide
segmented scan (Sec. 4.1: the filter is linear in (p_bar, L) with constant coefficients,
so consecutive updates of one pixel compose into one map).  Both must reproduce the
oracle: integer state bit-exactly, L, p_bar and images within 1e-4.  Streams dominated by
one hot pixel or one hot tile give chains of ~10^6 events, where the walk serialises and
the scan does not.
"""
import numpy as np
import pytest
import torch

import eventsim
from tests.harness import compare, plan_packets, run_gpu, run_oracle, sim

pytestmark = pytest.mark.gpu

MODES = {
    "nsf": dict(spatial_filter=0),
    "s1": dict(spatial_filter=1, blur_mode=0),
    "s2": dict(spatial_filter=1, blur_mode=1),
}
POLICY = {"auto": 0, "walk": 1, "scan": 2}


def _check(oracle_mod, W, H, ev, steps, mode, policy, **params):
    p = dict(MODES[mode], **params)
    o_imgs, o_states = run_oracle(oracle_mod, W, H, ev, steps, **p)
    g_imgs, g_states, stats = run_gpu(W, H, ev, steps, chain_policy=POLICY[policy], **p)
    worst = compare(W, H, o_imgs, o_states, g_imgs, g_states, spatial=p.get("spatial_filter", 1) == 1)
    return worst, stats


@pytest.mark.parametrize("policy", ["walk", "scan"])
@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_schedules_on_small_and_ragged_streams(oracle_mod, mode, policy):
    for (W, H, n, seed) in [(4, 4, 300, 1), (1, 1, 50, 5), (5, 3, 400, 4), (33, 17, 5000, 7)]:
        ev = eventsim.random_events(W, H, n, seed=seed)
        _, stats = _check(oracle_mod, W, H, ev, plan_packets(n, 97, 250, ev), mode, policy, q_min=1)
        key = "iir_scan_pieces" if policy == "scan" else "iir_walk_pieces"
        other = "iir_walk_pieces" if policy == "scan" else "iir_scan_pieces"
        assert stats[key] > 0 and stats[other] == 0, stats
    W, H = 96, 72
    ev = sim(W, H, 60_000, seed=3, noise=0.02)
    _check(oracle_mod, W, H, ev, plan_packets(60_000, 4093, 9_999, ev), mode, policy, c_on=0.2, c_off=0.2)


@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_scan_on_config_sine_checker_240x180_1M(oracle_mod, mode):
    """The scan on every piece of the full 240x180 stream (one read-out of 1 M events)."""
    ev = eventsim.make_config("sine_checker_240x180_1M")
    steps = [("push", 0, 1_000_000), ("read", int(ev[-1, 1]))]
    worst, _ = _check(oracle_mod, 240, 180, ev, steps, mode, "scan", c_on=0.2, c_off=0.2)
    assert worst <= 1e-4


def test_gain_with_scan(oracle_mod):
    """Sec. 5.2 gains enter the scan's maps as the factor on Eq. 6."""
    from paper_2510_20071_gb300 import Fibar
    W, H, n = 40, 30, 30_000
    ev = eventsim.hot_pixel_events(W, H, n, seed=4, hot=[(7, 9)], hot_frac=0.5)
    gain = (0.5 + np.random.default_rng(3).random(W * H)).astype(np.float32)
    for mode in ["s1", "s2", "nsf"]:
        p = dict(MODES[mode], c_on=0.2, c_off=0.2)
        o = oracle_mod.Oracle(W, H, **p)
        o.set_gain(gain.astype(np.float64))
        f = Fibar(W, H, chain_policy=2, **p)
        f.set_pixel_gain(torch.from_numpy(gain))
        dev = ev.cuda()
        for lo in range(0, n, 7_000):
            hi = min(n, lo + 7_000)
            o.push(ev[lo:hi])
            f.push(dev[lo:hi])
            t = int(ev[hi - 1, 1])
            ref = o.readout(t)
            img = f.readout(t).cpu().numpy()
            assert np.abs(img - ref).max() <= 1e-4
        f.close()
        o.close()


@pytest.mark.parametrize("hot", [[(17, 33)], [(40, 60), (41, 60), (40, 61), (41, 61)]],
                         ids=["one_pixel", "one_tile"])
@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_hot_streams_all_schedules(oracle_mod, mode, hot):
    """1 M events, 90 % of them on one pixel (or the four pixels of one tile), the rest
    uniform: every schedule matches the oracle, and auto picks the scan."""
    W, H, n = 240, 180, 1_000_000
    ev = eventsim.hot_pixel_events(W, H, n, seed=21, hot=hot, hot_frac=0.9)
    steps = plan_packets(n, 65_536, 250_000, ev)
    p = dict(MODES[mode], c_on=0.2, c_off=0.2)
    o_imgs, o_states = run_oracle(oracle_mod, W, H, ev, steps, **p)
    for policy in ["walk", "scan", "auto"]:
        g_imgs, g_states, stats = run_gpu(W, H, ev, steps, chain_policy=POLICY[policy], **p)
        compare(W, H, o_imgs, o_states, g_imgs, g_states, spatial=p.get("spatial_filter", 1) == 1)
        if policy == "walk":
            assert stats["iir_scan_pieces"] == 0
        else:
            assert stats["iir_scan_pieces"] > 0, stats


def _walk_ms(ev, policy, W, H, batches, per_batch):
    from paper_2510_20071_gb300 import Fibar
    f = Fibar(W, H, chain_policy=POLICY[policy], c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=1)
    dev = ev.cuda()
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    imgs = []
    for b in range(batches):
        if b == 1:
            f.stage_times(reset=True)
            f.set_timing(True)
        lo, hi = b * per_batch, (b + 1) * per_batch
        f.push(dev[lo:hi])
        f.readout(int(ev[hi - 1, 1]), out)
        imgs.append(out.cpu().numpy().copy())
    st = f.stage_times(reset=True)
    f.close()
    return st["walk"] / max(st["calls"], 1), imgs


def test_scan_at_least_10x_faster_than_walk_on_a_hot_tile():
    """All 1 M events of each read-out on the four pixels of one tile: the walk runs each
    piece's chain in one thread, the scan in a few block-wide levels."""
    W, H, per = 240, 180, 1_000_000
    ev = eventsim.hot_pixel_events(W, H, 4 * per, seed=22, hot=[(100, 50), (101, 50), (100, 51), (101, 51)],
                                   hot_frac=1.0)
    t_walk, img_w = _walk_ms(ev, "walk", W, H, 4, per)
    t_scan, img_s = _walk_ms(ev, "scan", W, H, 4, per)
    for a, b in zip(img_w, img_s):
        assert np.abs(a - b).max() <= 1e-4
    print(f"walk stage: walk {t_walk:.3f} ms, scan {t_scan:.3f} ms per 1 M-event read-out")
    assert t_walk >= 10.0 * t_scan, (t_walk, t_scan)

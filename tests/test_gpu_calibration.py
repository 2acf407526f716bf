"""GPU parity of the threshold calibration (fibar_relative_thresholds) and of the Sec. 5.2
correction (fibar_set_pixel_gain) against the FP64 oracle."""
import ctypes as C

import numpy as np
import pytest
import torch

import eventsim
import oracle
from tests.harness import compare, plan_packets

pytestmark = pytest.mark.gpu

MODES = {
    "nsf": dict(spatial_filter=0),
    "s1": dict(spatial_filter=1, blur_mode=0),
    "s2": dict(spatial_filter=1, blur_mode=1),
}


def _rel_close(got, exp):
    """float32 quotients of exact counts: within a few float32 ulps; NaN where the oracle
    has NaN."""
    got = got.astype(np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(exp))
    m = ~np.isnan(exp)
    np.testing.assert_allclose(got[m], exp[m], rtol=3e-7, atol=0)


@pytest.mark.parametrize("device", [True, False])
def test_relative_thresholds_match_oracle(device):
    from paper_2510_20071_gb300 import relative_thresholds
    r = eventsim.threshold_recording(64, 48, periods=6, amplitude=8.0, steps_per_half=160)
    ev = r["events"]
    # add records outside the sensor and leave some pixels without events
    extra = eventsim.pack_events(torch.tensor([64, 3, 70]), torch.tensor([0, 48, 50]),
                                 torch.tensor([1, -1, 1]), torch.tensor([0, 0, 0]))
    keep = (ev[:, 0] & 0xFFFF) >= 4  # pixels in columns 0..3 get no events
    ev = torch.cat([ev[keep], extra]).contiguous()
    exp = oracle.relative_thresholds(64, 48, ev)
    got = relative_thresholds(ev.cuda() if device else ev, 64, 48)
    for g, e in zip(got, exp):
        _rel_close(g.cpu().numpy(), e)


def test_relative_thresholds_large_and_empty():
    from paper_2510_20071_gb300 import relative_thresholds, binding
    W, H = 640, 480
    ev = eventsim.random_events(W, H, 3_000_000, seed=2, p_on=0.55)
    exp = oracle.relative_thresholds(W, H, ev)
    got = relative_thresholds(ev.cuda(), W, H)
    for g, e in zip(got, exp):
        _rel_close(g.cpu().numpy(), e)
    # host path in several staged chunks would need > 4 Mi records; one chunk here
    got_h = relative_thresholds(ev, W, H)
    for g, e in zip(got_h, exp):
        _rel_close(g.numpy(), e)
    # no events: every value undefined
    empty = torch.zeros((0, 2), dtype=torch.int64)
    for g in relative_thresholds(empty.cuda(), 8, 4):
        assert torch.isnan(g).all()
    # bad arguments
    outs = [torch.empty(4, device="cuda") for _ in range(3)]
    assert binding.fibar_relative_thresholds(None, 5, 2, 2, 1, *[o.data_ptr() for o in outs], 0) != 0
    assert binding.fibar_relative_thresholds(None, 0, 0, 2, 1, *[o.data_ptr() for o in outs], 0) != 0


def _gained_run(mode, W, H, ev, steps, gain, device_gain):
    from paper_2510_20071_gb300 import Fibar
    params = dict(MODES[mode], c_on=0.2, c_off=0.2)
    o = oracle.Oracle(W, H, **params)
    o.set_gain(gain.astype(np.float32).astype(np.float64))
    f = Fibar(W, H, **params)
    g = torch.from_numpy(gain.astype(np.float32))
    f.set_pixel_gain(g.cuda() if device_gain else g)
    ev_dev = ev.cuda()
    o_imgs, o_states, g_imgs, g_states = [], [], [], []
    for st in steps:
        if st[0] == "push":
            o.push(ev[st[1]:st[2]])
            f.push(ev_dev[st[1]:st[2]])
        else:
            o_imgs.append(o.readout(st[1]))
            o_states.append(o.state())
            g_imgs.append(f.readout(st[1]).cpu().numpy().astype(np.float64))
            g_states.append(f.state())
    f.close()
    o.close()
    return o_imgs, o_states, g_imgs, g_states


@pytest.mark.parametrize("mode", ["s2", "s1", "nsf"])
def test_gain_correction_matches_oracle(mode):
    W, H = 96, 72
    ev = eventsim.simulate(W, H, 60_000, scene="sine_checker", seed=3, noise_frac=0.02)
    steps = plan_packets(60_000, 4093, 9_999, ev)
    # gains from a calibration of the same sensor size (relative thresholds C'_i)
    r = eventsim.threshold_recording(W, H, periods=4, amplitude=4.0, steps_per_half=80, seed=8)
    c = oracle.relative_thresholds(W, H, r["events"])[2].ravel()
    c = np.where(np.isnan(c), 1.0, c)
    o_imgs, o_states, g_imgs, g_states = _gained_run(mode, W, H, ev, steps, c, device_gain=(mode != "nsf"))
    compare(W, H, o_imgs, o_states, g_imgs, g_states, spatial=MODES[mode].get("spatial_filter", 1) == 1)


def test_gain_validation_and_removal():
    from paper_2510_20071_gb300 import Fibar, FibarError
    W, H = 16, 8
    f = Fibar(W, H, c_on=0.2, c_off=0.2)
    bad = torch.ones(W * H)
    bad[5] = 0.0
    with pytest.raises(FibarError):
        f.set_pixel_gain(bad)
    with pytest.raises(TypeError):
        f.set_pixel_gain(torch.ones(W * H - 1))
    ev = eventsim.random_events(W, H, 3000, seed=1)
    f.set_pixel_gain(torch.full((W * H,), 2.0))
    f.set_pixel_gain(None)  # removed: the plain filter
    f.push(ev.cuda())
    got = f.readout(int(ev[-1, 1])).cpu().numpy()
    o = oracle.Oracle(W, H, c_on=0.2, c_off=0.2)
    o.push(ev)
    np.testing.assert_allclose(got, o.readout(int(ev[-1, 1])), atol=1e-4, rtol=0)
    f.close()

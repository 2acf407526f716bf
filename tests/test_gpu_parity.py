"""GPU parity: the CUDA library against the FP64 oracle on the same seeded streams.

Integer state (events applied, queue window h/q, q_targ, N_ap, N_at, per-pixel queued
counts, per-tile active counts, stale masks, last event index) must match bit-exactly;
L, p_bar and read-out images within 1e-4 absolute (log brightness at C = 0.2).
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


def _check(oracle_mod, W, H, ev, steps, mode, device_push=True, host_out=False, **params):
    p = dict(MODES[mode])
    p.update(params)
    o_imgs, o_states = run_oracle(oracle_mod, W, H, ev, steps, **p)
    g_imgs, g_states, stats = run_gpu(W, H, ev, steps, device_push=device_push, host_out=host_out, **p)
    worst = compare(W, H, o_imgs, o_states, g_imgs, g_states, spatial=p.get("spatial_filter", 1) == 1)
    return worst, stats


@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_small_random_streams(oracle_mod, mode):
    for (W, H, n, seed) in [(4, 4, 300, 1), (6, 4, 500, 2), (8, 8, 2000, 3), (5, 3, 400, 4),
                            (1, 1, 50, 5), (2, 2, 100, 6), (33, 17, 5000, 7)]:
        ev = eventsim.random_events(W, H, n, seed=seed)
        steps = plan_packets(n, 97, 250, ev)
        _check(oracle_mod, W, H, ev, steps, mode, q_min=1)


@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_sine_checker_several_tiles_and_ragged_tail(oracle_mod, mode):
    W, H = 96, 72
    ev = sim(W, H, 60_000, seed=3, noise=0.02)
    steps = plan_packets(60_000, 4093, 9_999, ev)
    _check(oracle_mod, W, H, ev, steps, mode, c_on=0.2, c_off=0.2)


def test_config_sine_checker_240x180_1M_full(oracle_mod):
    """240x180, 1,000,000 events, translating sinusoid+checker, seed 0, one read-out."""
    ev = eventsim.make_config("sine_checker_240x180_1M")
    steps = [("push", 0, 1_000_000), ("read", int(ev[-1, 1]))]
    for mode in ["nsf", "s1", "s2"]:
        worst, stats = _check(oracle_mod, 240, 180, ev, steps, mode, c_on=0.2, c_off=0.2)
        assert worst <= 1e-4


def test_config_perlin_1280x720_prefix(oracle_mod):
    """1280x720 rotating+zooming Perlin with 2% noise events, 65,536-event packets and a
    read-out every 1,000,000 events (first 3 M events of the stream)."""
    n = 3_000_000
    ev = eventsim.make_config("perlin_1280x720_200M", n_events=n, device="cuda").cpu()
    steps = plan_packets(n, 65_536, 1_000_000, ev)
    for mode in ["s2", "s1"]:
        _, stats = _check(oracle_mod, 1280, 720, ev, steps, mode, c_on=0.2, c_off=0.2)
        # the speculative detector's guesses hold from the first read-out on (the queue
        # grows from empty to ~36,000 events in it): the serial fixup reruns few events
        assert stats["detector_fix_steps"] < n // 100, stats


@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_host_push_and_host_readout(oracle_mod, mode):
    W, H = 40, 30
    ev = sim(W, H, 20_000, seed=9)
    steps = plan_packets(20_000, 3000, 7000, ev)
    _check(oracle_mod, W, H, ev, steps, mode, device_push=False, host_out=True, c_on=0.2, c_off=0.2)


def test_readout_mid_packet_and_nonmonotone_time(oracle_mod):
    W, H = 24, 20
    ev = eventsim.random_events(W, H, 3000, seed=11, t_step_us=3)
    ev[1500, 1] = 10**9  # a late record blocks everything after it until a later read-out
    steps = [("push", 0, 1000), ("read", 700), ("push", 1000, 3000), ("read", 2000),
             ("read", 2000), ("read", 5000), ("read", 10**9), ("read", 10**10)]
    for mode in ["nsf", "s1", "s2"]:
        _check(oracle_mod, W, H, ev, steps, mode, q_min=1)


def test_out_of_range_events_dropped(oracle_mod):
    W, H = 16, 12
    ev = eventsim.random_events(W, H, 2000, seed=12)
    bad = eventsim.pack_events(torch.tensor([16, 3, 200, 0]), torch.tensor([0, 12, 5, 65535]),
                               torch.tensor([1, -1, 1, 1]), torch.tensor([0, 0, 0, 0]))
    ev = torch.cat([ev[:500], bad, ev[500:1500], bad, ev[1500:]])
    ev[:, 1] = torch.arange(ev.shape[0])
    steps = plan_packets(ev.shape[0], 333, 800, ev)
    _, _, stats = run_gpu(W, H, ev, steps, **MODES["s2"])
    assert stats["events_dropped"] == 8 and stats["events_applied"] == 2000
    _check(oracle_mod, W, H, ev, steps, "s2")


def test_packet_split_invariance(oracle_mod):
    W, H = 48, 36
    ev = sim(W, H, 30_000, seed=13, noise=0.05)
    # single-event packets (host pushes coalesce in the staging buffer)
    sub = 3000
    steps = plan_packets(sub, 1, 700, ev[:sub])
    imgs, states, _ = run_gpu(W, H, ev[:sub], steps, device_push=False, **MODES["s2"])
    o_imgs, o_states = run_oracle(oracle_mod, W, H, ev[:sub], steps, **MODES["s2"])
    compare(W, H, o_imgs, o_states, imgs, states)
    # device packets of several sizes: identical results
    results = []
    for packet in [977, 8192, 30_000]:
        steps = plan_packets(30_000, packet, None, ev)
        imgs, states, _ = run_gpu(W, H, ev, steps, **MODES["s2"])
        results.append((imgs[-1], states[-1]))
    for img, st in results[1:]:
        np.testing.assert_array_equal(img, results[0][0])
        for key in ["h", "q_targ", "n_ap", "n_at"]:
            assert st[key] == results[0][1][key]
        np.testing.assert_array_equal(st["cnt"], results[0][1]["cnt"])


def test_pending_device_packet_limit():
    from paper_2510_20071_gb300 import FibarError, FIBAR_ENOMEM, Fibar
    ev = eventsim.random_events(8, 8, 300, seed=1).cuda()
    f = Fibar(8, 8)
    for i in range(192):
        f.push(ev[i:i + 1])
    with pytest.raises(FibarError) as e:
        f.push(ev[192:193])
    assert e.value.code == FIBAR_ENOMEM
    f.readout(10**9)
    f.push(ev[192:193])  # accepted again after the read-out
    f.flush()
    assert f.stats()["events_applied"] == 193
    f.close()


@pytest.mark.parametrize("params", [dict(q_min=1), dict(q_min=7, q_init=50), dict(fill_num=7, fill_den=10),
                                    dict(fill_num=1, fill_den=4), dict(t_cut=float("inf")),
                                    dict(t_cut=100.0, c_on=0.25, c_off=0.35)])
def test_parameter_variants(oracle_mod, params):
    W, H = 30, 22
    ev = sim(W, H, 25_000, seed=14, noise=0.03)
    steps = plan_packets(25_000, 5000, 6000, ev)
    _check(oracle_mod, W, H, ev, steps, "s2", **params)
    _check(oracle_mod, W, H, ev, steps, "s1", **params)


def test_degenerate_streams(oracle_mod):
    # one pixel only (one tile holds every event: one long segment), one tile cycling,
    # an empty read-out, and a push of zero events
    W, H = 64, 64
    for pixels in [[1000], [0, 1, 64, 65], [4095]]:
        ev = eventsim.random_events(W, H, 20_000, seed=15, pixels=pixels)
        steps = [("read", 0), ("push", 0, 0), ("push", 0, 20_000), ("read", 10**12)]
        _check(oracle_mod, W, H, ev, steps, "s2", q_min=1)
        _check(oracle_mod, W, H, ev, steps, "s1", q_min=1)
        _check(oracle_mod, W, H, ev, steps, "nsf")


def test_large_batch_many_chunks(oracle_mod):
    """One read-out over 4 M events (16 k detector chunks) on 640x480."""
    W, H = 640, 480
    n = 4_000_000
    ev = eventsim.simulate(W, H, n, scene=eventsim.SceneSpec(texture="perlin"), seed=21,
                           noise_frac=0.02, device="cuda").cpu()
    steps = [("push", 0, n), ("read", int(ev[-1, 1]))]
    _check(oracle_mod, W, H, ev, steps, "s2", c_on=0.2, c_off=0.2)
    _check(oracle_mod, W, H, ev, steps, "s1", c_on=0.2, c_off=0.2)


def _swing_stream(W, H, phases, seed):
    """Alternating phases: uniform pixels (mostly distinct tiles: Eq. 20 doubles the
    target) and all four pixels of a few tiles (r = 1: the target halves), so the queue
    length swings by orders of magnitude inside one batch."""
    parts, t0 = [], 0
    dense = np.array([(ty * 2 + dy) * W + tx * 2 + dx for ty in range(8) for tx in range(8)
                      for dy in range(2) for dx in range(2)])
    for i, (kind, n) in enumerate(phases):
        ev = eventsim.random_events(W, H, n, seed=seed + i, pixels=dense if kind == "dense" else None)
        ev[:, 1] += t0
        t0 = int(ev[-1, 1]) + 1
        parts.append(ev)
    return torch.cat(parts)


@pytest.mark.parametrize("mode", ["s2", "s1"])
def test_queue_swings_within_a_batch(oracle_mod, mode):
    """Inside one read-out the queue grows from ~40,000 events to the sensor size
    (65,536) and back, and in the next it falls to ~170 and rises to ~40,000 again, so
    the detector's window guesses fall outside the window table's band."""
    W, H = 256, 256
    ev = _swing_stream(W, H, [("spread", 150_000), ("dense", 60_000), ("spread", 200_000),
                              ("dense", 150_000), ("spread", 100_000)], seed=31)
    n = ev.shape[0]
    steps = [("push", 0, 300_000), ("read", int(ev[299_999, 1])), ("push", 300_000, n),
             ("read", int(ev[-1, 1]))]
    _check(oracle_mod, W, H, ev, steps, mode, q_min=4)


def test_determinism(oracle_mod):
    W, H = 64, 48
    ev = sim(W, H, 50_000, seed=16, noise=0.02)
    steps = plan_packets(50_000, 8192, 12_000, ev)
    for mode in ["s1", "s2"]:
        a = run_gpu(W, H, ev, steps, **MODES[mode])
        b = run_gpu(W, H, ev, steps, **MODES[mode])
        for x, y in zip(a[0], b[0]):
            np.testing.assert_array_equal(x, y)


def test_bounded_device_wait_reports_timeout_and_handle_recovers(oracle_mod):
    """A bounded device wait on a flag that nothing sets gives up after its poll limit and
    the host reads ETIMEOUT (no trap, no hang); the handle keeps working afterwards."""
    from paper_2510_20071_gb300 import Fibar, FIBAR_ETIMEOUT, binding
    W, H = 32, 24
    ev = eventsim.random_events(W, H, 4000, seed=12)
    f = Fibar(W, H, spatial_filter=1, blur_mode=1, q_min=4)
    try:
        f.push(ev[:2000].cuda())
        f.readout(int(ev[1999, 1]))
        rc = binding.fibar_debug_wait_timeout(f.h, 2000, f._s)
        assert rc == FIBAR_ETIMEOUT
        assert "gave up" in binding.fibar_last_error(f.h)
        assert binding.fibar_debug_wait_timeout(f.h, 0, f._s) == binding.FIBAR_EINVAL
        f.push(ev[2000:].cuda())
        out = torch.empty((H, W), dtype=torch.float32).pin_memory()
        f.readout(int(ev[-1, 1]), out)  # host read-out checks the error flags: none left
        o = oracle_mod.Oracle(W, H, spatial_filter=1, blur_mode=1, q_min=4)
        o.push(ev[:2000]); o.readout(int(ev[1999, 1])); o.push(ev[2000:])
        np.testing.assert_allclose(out.numpy(), o.readout(int(ev[-1, 1])), atol=1e-4, rtol=0)
        assert f.stats()["events_applied"] == 4000
    finally:
        f.close()


@pytest.mark.parametrize("device", [True, False])
def test_push_many_equals_single_pushes(device):
    """fibar_push_events_many (adjacent packets merged into one copy or segment, others kept
    apart) gives the same images and state as one fibar_push_events per packet."""
    from paper_2510_20071_gb300 import Fibar
    W, H = 64, 48
    ev = eventsim.random_events(W, H, 30_000, seed=17)
    other = eventsim.random_events(W, H, 30_000, seed=18)  # a second buffer: not adjacent
    src = (ev.cuda(), other.cuda()) if device else (ev.pin_memory(), other.pin_memory())
    cuts = [0, 3000, 3001, 9000, 15000, 15000, 22000, 30000]
    packets = [(0, a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
    # a copy of one packet from the other buffer (same records) breaks adjacency
    mixed = []
    for i, (_, a, b) in enumerate(packets):
        if i == 2:
            alt = src[1][:b - a]
            alt.copy_(src[0][a:b])
            mixed.append(alt)
        else:
            mixed.append(src[0][a:b])
    t_mid, t_end = int(ev[14_999, 1]), int(ev[-1, 1])
    outs = []
    for many in (False, True):
        f = Fibar(W, H, spatial_filter=1, blur_mode=1, q_min=4)
        if many:
            f.push_many(mixed[:3])
            imgs = [f.readout(t_mid).cpu()]
            f.push_many(mixed[3:])
        else:
            for p in mixed[:3]:
                f.push(p)
            imgs = [f.readout(t_mid).cpu()]
            for p in mixed[3:]:
                f.push(p)
        imgs.append(f.readout(t_end).cpu())
        st = f.state()
        outs.append((imgs, st))
        f.close()
    (a_imgs, a_st), (b_imgs, b_st) = outs
    for x, y in zip(a_imgs, b_imgs):
        assert torch.equal(x, y)
    for k in ["k", "h", "q", "q_targ", "n_ap", "n_at"]:
        assert a_st[k] == b_st[k]
    np.testing.assert_array_equal(a_st["L"], b_st["L"])
    np.testing.assert_array_equal(a_st["cnt"], b_st["cnt"])


PAN_PREFIX = 20_000_000


@pytest.fixture(scope="module")
def pan_prefix():
    return eventsim.make_config("perlin_pan_1280x720_1B", n_events=PAN_PREFIX, device="cuda").cpu()


@pytest.mark.parametrize("packet", [8_192, 65_536, 1_048_576])
def test_config_perlin_pan_1280x720_prefix(oracle_mod, pan_prefix, packet):
    """1280x720 Perlin noise panned in bursts (segments of 1-50 Mev/s), seed 2: the first
    20 M events, read out every 1,000,000 events, pushed as packets of 8,192, 65,536 and
    1,048,576 events (S2).  The temporal filter's schedule is chosen per piece (auto)."""
    n = PAN_PREFIX
    ev = pan_prefix
    steps = plan_packets(n, packet, 1_000_000, ev)
    worst, stats = _check(oracle_mod, 1280, 720, ev, steps, "s2", c_on=0.2, c_off=0.2)
    assert stats["events_applied"] == n
    print(f"packet {packet}: max |diff| {worst:.2e}, walk pieces {stats['iir_walk_pieces']}, "
          f"scan pieces {stats['iir_scan_pieces']}, fixup steps {stats['detector_fix_steps']}")


@pytest.mark.parametrize("mode", ["nsf", "s1", "s2"])
def test_pinned_host_push_and_async_host_readout(oracle_mod, mode):
    """Host packets from page-locked memory (copied on the handle's copy stream into two
    alternating staging buffers) and fibar_readout_host_async images, waited for once at
    the end: every image equals the oracle's."""
    from paper_2510_20071_gb300 import Fibar
    W, H, n = 64, 48, 40_000
    ev = sim(W, H, n, seed=19, noise=0.01)
    steps = plan_packets(n, 3_000, 7_000, ev)
    p = dict(MODES[mode], c_on=0.2, c_off=0.2)
    o_imgs, o_states = run_oracle(oracle_mod, W, H, ev, steps, **p)
    host = ev.pin_memory()
    bufs = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in o_imgs]
    f = Fibar(W, H, **p)
    r = 0
    for st in steps:
        if st[0] == "push":
            f.push(host[st[1]:st[2]])
        else:
            f.readout_host_async(st[1], bufs[r])
            r += 1
    f.wait()
    g_state = f.state()
    f.close()
    for i, (a, b) in enumerate(zip(o_imgs, bufs)):
        assert np.abs(a - b.numpy()).max() <= 1e-4, i
    assert g_state["k"] == o_states[-1]["k"]
    if p.get("spatial_filter", 1):
        for key in ["h", "q_targ", "n_ap", "n_at"]:
            assert g_state[key] == o_states[-1][key]

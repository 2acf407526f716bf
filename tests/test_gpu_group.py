"""Group read-outs (fibar_group_*: every member's read-out chain captured once into a CUDA
graph launched on the member's own stream) on the GPU: bit-identical to the same handles
read out one call at a time, argument checks that leave the members untouched, re-capture
after a member's configuration changes, host packets, the descriptor ring wrapping, and
latency stamps."""
import numpy as np
import pytest
import torch

import eventsim

pytestmark = pytest.mark.gpu

SENSORS = [(64, 48), (96, 72), (120, 90), (33, 17)]
MODES = {
    "nsf": dict(spatial_filter=0),
    "s1": dict(spatial_filter=1, blur_mode=0),
    "s2": dict(spatial_filter=1, blur_mode=1),
}


def _streams(n, seed, events=60_000):
    out = []
    for i in range(n):
        W, H = SENSORS[i % len(SENSORS)]
        ev = eventsim.simulate(W, H, events + 7919 * i, scene="perlin", seed=seed + i, noise_frac=0.02)
        out.append((W, H, ev.cuda()))
    return out


def _pair(streams, params):
    from paper_2510_20071_gb300 import Fibar
    a = [Fibar(W, H, **params) for W, H, _ in streams]
    b = [Fibar(W, H, **params) for W, H, _ in streams]
    return a, b


def _close(*fibs):
    for fs in fibs:
        for f in fs:
            f.close()


def _out(f):
    return torch.empty((f.H, f.W), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("mode", ["s2", "s1", "nsf"])
def test_group_matches_direct_readouts_bit_for_bit(mode):
    from paper_2510_20071_gb300 import Group
    params = dict(MODES[mode], c_on=0.2, c_off=0.2)
    streams = _streams(5, seed=51)
    direct, grouped = _pair(streams, params)
    g = Group(grouped)
    rng = np.random.default_rng(5)
    pos = [0] * len(streams)
    try:
        for rnd in range(6):
            # a random subset of the members each round, several packets each
            members = sorted(rng.choice(len(streams), size=rng.integers(1, len(streams) + 1), replace=False))
            ts, outs_d, outs_g = [], [], []
            for i in members:
                ev = streams[i][2]
                hi = min(ev.shape[0], pos[i] + int(rng.integers(3000, 12000)))
                for lo in range(pos[i], hi, 2500):
                    pk = ev[lo:min(hi, lo + 2500)]
                    direct[i].push(pk)
                    grouped[i].push(pk)
                pos[i] = hi
                t = int(ev[hi - 1, 1].item())
                ts.append(t)
                outs_d.append(direct[i].readout(t))
                outs_g.append(_out(grouped[i]))
            g.readout([int(i) for i in members], ts, outs_g)
            torch.cuda.synchronize()
            for i, a, b in zip(members, outs_d, outs_g):
                assert torch.equal(a, b), f"round {rnd}, member {i}"
        for fd, fg in zip(direct, grouped):
            sd, sg = fd.state(), fg.state()
            for k in sd:
                np.testing.assert_array_equal(np.asarray(sd[k]), np.asarray(sg[k]), err_msg=k)
            assert fd.stats()["events_applied"] == fg.stats()["events_applied"]
        st = g.stats()
        assert st["members"] == len(streams) and st["graph_launches"] == 6 and st["builds"] == len(streams)
    finally:
        g.close()
        _close(direct, grouped)


def test_group_checks_leave_members_untouched():
    from paper_2510_20071_gb300 import FibarError, FIBAR_EINVAL, FIBAR_EORDER, Group
    params = dict(spatial_filter=1, blur_mode=1, c_on=0.2, c_off=0.2)
    streams = _streams(3, seed=61, events=20_000)
    direct, grouped = _pair(streams, params)
    g = Group(grouped)
    try:
        for i, (_, _, ev) in enumerate(streams):
            direct[i].push(ev[:10_000])
            grouped[i].push(ev[:10_000])
        t = [int(ev[9_999, 1].item()) for _, _, ev in streams]
        outs = [_out(f) for f in grouped]
        ref = [direct[i].readout(t[i]) for i in range(3)]
        g.readout([0, 1, 2], t, outs)
        # repeated member, misaligned output, time going back: nothing is queued
        with pytest.raises(FibarError) as e:
            g.readout([0, 0], [t[0] + 1, t[0] + 2], [outs[0], outs[0]])
        assert e.value.code == FIBAR_EINVAL
        flat = torch.empty(grouped[1].W * grouped[1].H + 1, dtype=torch.float32, device="cuda")
        with pytest.raises(FibarError) as e:
            g.readout([1], [t[1] + 5], [flat[1:]])
        assert e.value.code == FIBAR_EINVAL
        with pytest.raises(FibarError) as e:
            g.readout([2, 1], [t[2] - 1, t[1] + 5], [outs[2], outs[1]])
        assert e.value.code == FIBAR_EORDER
        assert g.stats()["graph_launches"] == 1
        # the members carry on exactly like handles that never saw the failed calls
        for i, (_, _, ev) in enumerate(streams):
            direct[i].push(ev[10_000:20_000])
            grouped[i].push(ev[10_000:20_000])
        t2 = [int(ev[19_999, 1].item()) for _, _, ev in streams]
        torch.cuda.synchronize()
        for i in range(3):
            assert torch.equal(ref[i], outs[i])
        ref2 = [direct[i].readout(t2[i]) for i in range(3)]
        outs2 = [_out(f) for f in grouped]
        g.readout([2, 0, 1], [t2[2], t2[0], t2[1]], [outs2[2], outs2[0], outs2[1]])
        torch.cuda.synchronize()
        for i in range(3):
            assert torch.equal(ref2[i], outs2[i])
    finally:
        g.close()
        _close(direct, grouped)


def test_group_recaptures_after_a_member_changes():
    from paper_2510_20071_gb300 import Group
    params = dict(spatial_filter=1, blur_mode=1, c_on=0.2, c_off=0.2)
    streams = _streams(2, seed=71, events=30_000)
    direct, grouped = _pair(streams, params)
    g = Group(grouped)
    try:
        for step, (lo, hi) in enumerate([(0, 10_000), (10_000, 20_000), (20_000, 30_000)]):
            if step == 1:
                for f in direct + grouped:
                    f.set_grid_share(3)
            if step == 2:
                gain = (0.5 + torch.rand(streams[0][1] * streams[0][0], generator=torch.Generator().manual_seed(3)))
                direct[0].set_pixel_gain(gain.cuda())
                grouped[0].set_pixel_gain(gain.cuda())
            ts, outs = [], []
            for i, (_, _, ev) in enumerate(streams):
                direct[i].push(ev[lo:hi])
                grouped[i].push(ev[lo:hi])
                ts.append(int(ev[hi - 1, 1].item()))
                outs.append(_out(grouped[i]))
            ref = [direct[i].readout(ts[i]) for i in range(2)]
            g.readout([0, 1], ts, outs)
            torch.cuda.synchronize()
            for i in range(2):
                assert torch.equal(ref[i], outs[i]), (step, i)
        # one capture per member, then both after the grid share, member 0 after its gains
        assert g.stats()["builds"] == 2 + 2 + 1
    finally:
        g.close()
        _close(direct, grouped)


def test_group_with_host_packets_and_latency_stamps():
    from paper_2510_20071_gb300 import Group
    params = dict(spatial_filter=1, blur_mode=1, c_on=0.2, c_off=0.2)
    streams = _streams(3, seed=81, events=40_000)
    direct, grouped = _pair(streams, params)
    g = Group(grouped)
    try:
        tickets = []
        for lo, hi in [(0, 15_000), (15_000, 40_000)]:
            ts, outs = [], []
            for i, (_, _, ev) in enumerate(streams):
                host = ev[lo:hi].cpu().pin_memory()
                direct[i].push(host)
                grouped[i].push(host)
                ts.append(int(ev[hi - 1, 1].item()))
                outs.append(_out(grouped[i]))
            ref = [direct[i].readout(ts[i]) for i in range(3)]
            tickets.append(g.readout([0, 1, 2], ts, outs))
            torch.cuda.synchronize()
            for i in range(3):
                assert torch.equal(ref[i], outs[i])
        for tk in tickets:
            lat = g.latency_ms(tk, 3)
            assert all(0.0 < x < 1000.0 for x in lat), lat
    finally:
        g.close()
        _close(direct, grouped)


def test_group_learned_fill_member():
    from paper_2510_20071_gb300 import Group
    from paper_2510_20071_gb300.fill import init_params
    params = dict(spatial_filter=1, blur_mode=2, c_on=0.2, c_off=0.2)
    W, H = 300, 140
    ev = eventsim.simulate(W, H, 200_000, scene="perlin", seed=91, noise_frac=0.02).cuda()
    from paper_2510_20071_gb300 import Fibar
    fd, fg = Fibar(W, H, **params), Fibar(W, H, **params)
    theta = init_params(4).astype(np.float32)
    fd.set_fill_weights(theta)
    fg.set_fill_weights(theta)
    g = Group([fg])
    try:
        for lo, hi in [(0, 120_000), (120_000, 200_000)]:
            fd.push(ev[lo:hi])
            fg.push(ev[lo:hi])
            t = int(ev[hi - 1, 1].item())
            out = _out(fg)
            ref = fd.readout(t)
            g.readout([0], [t], [out])
            torch.cuda.synchronize()
            assert torch.equal(ref, out)
    finally:
        g.close()
        fd.close()
        fg.close()


def test_group_descriptor_ring_wraps_without_waiting():
    """40 read-outs of each member queued back to back (more than the 16 descriptor slots
    per member), then compared with the same read-outs done directly."""
    from paper_2510_20071_gb300 import Group
    params = dict(spatial_filter=1, blur_mode=1, c_on=0.2, c_off=0.2)
    streams = _streams(2, seed=101, events=80_000)
    direct, grouped = _pair(streams, params)
    g = Group(grouped)
    try:
        outs_g, outs_d = [], []
        for r in range(40):
            lo, hi = 2000 * r, 2000 * (r + 1)
            ts, og = [], []
            for i, (_, _, ev) in enumerate(streams):
                direct[i].push(ev[lo:hi])
                grouped[i].push(ev[lo:hi])
                ts.append(int(ev[hi - 1, 1].item()))
                og.append(_out(grouped[i]))
                outs_d.append(direct[i].readout(ts[-1]))
            g.readout([0, 1], ts, og)
            outs_g.extend(og)
        g.join()
        torch.cuda.synchronize()
        for a, b in zip(outs_d, outs_g):
            assert torch.equal(a, b)
    finally:
        g.close()
        _close(direct, grouped)

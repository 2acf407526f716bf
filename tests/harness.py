"""Drive the CUDA library and the FP64 oracle identically on one event stream.

A run is a list of steps: ("push", lo, hi) pushes events [lo, hi) as one packet,
("read", t_us) reads out at t_us, ("flush",) applies everything pending.  Both sides
record every read-out image and the state after it.
"""
from __future__ import annotations

import numpy as np
import torch

import eventsim

LOG_TOL = 1e-4  # absolute, per pixel, in the units of L (log brightness when C = 0.2)


def plan_packets(n: int, packet: int, read_every: int | None, ev: torch.Tensor | None = None,
                 read_times: list[int] | None = None):
    """Push packets of `packet` events; read out after every `read_every` events (at the
    time stamp of the last event of that block) and once at the end."""
    steps = []
    tcol = ev[:, 1] if ev is not None else None
    next_read = read_every if read_every else None
    pos = 0
    while pos < n:
        hi = min(n, pos + packet)
        steps.append(("push", pos, hi))
        pos = hi
        while next_read is not None and next_read <= pos:
            steps.append(("read", int(tcol[next_read - 1])))
            next_read += read_every
    if read_times:
        for t in read_times:
            steps.append(("read", int(t)))
    steps.append(("read", int(tcol[-1]) if n else 0))
    return steps


def run_oracle(oracle_mod, W, H, ev, steps, **params):
    o = oracle_mod.Oracle(W, H, **params)
    imgs, states = [], []
    for st in steps:
        if st[0] == "push":
            o.push(ev[st[1]:st[2]])
        elif st[0] == "read":
            imgs.append(o.readout(st[1]))
            states.append(o.state())
        else:
            o.flush()
            states.append(o.state())
    return imgs, states


def run_gpu(W, H, ev, steps, device_push=True, host_out=False, **params):
    from paper_2510_20071_gb300 import Fibar
    f = Fibar(W, H, **params)
    ev_dev = ev.cuda() if device_push else ev
    imgs, states = [], []
    try:
        for st in steps:
            if st[0] == "push":
                f.push(ev_dev[st[1]:st[2]])
            elif st[0] == "read":
                if host_out:
                    out = torch.empty((H, W), dtype=torch.float32).pin_memory()
                    f.readout(st[1], out)
                    imgs.append(out.numpy().astype(np.float64))
                else:
                    imgs.append(f.readout(st[1]).cpu().numpy().astype(np.float64))
                states.append(f.state())
            else:
                f.flush()
                states.append(f.state())
        stats = f.stats()
    finally:
        f.close()
    return imgs, states, stats


def compare(W, H, o_imgs, o_states, g_imgs, g_states, spatial=True, tol=LOG_TOL):
    """Integer state bit-exact, floating point within `tol` absolute."""
    assert len(o_imgs) == len(g_imgs)
    worst = 0.0
    for i, (oi, gi) in enumerate(zip(o_imgs, g_imgs)):
        d = np.abs(oi.reshape(H, W) - gi.reshape(H, W))
        worst = max(worst, float(d.max(initial=0.0)))
        assert d.max(initial=0.0) <= tol, f"read-out {i}: max |diff| {d.max()} > {tol}"
    for i, (os_, gs) in enumerate(zip(o_states, g_states)):
        assert gs["k"] == os_["k"], f"state {i}: events applied {gs['k']} != {os_['k']}"
        last_o = os_["last"].astype(np.uint64)
        np.testing.assert_array_equal(gs["last_idx"], last_o, err_msg=f"state {i}: last_idx")
        np.testing.assert_allclose(gs["L"], os_["L"], atol=tol, rtol=0, err_msg=f"state {i}: L")
        np.testing.assert_allclose(gs["pbar"], os_["pbar"], atol=tol, rtol=0, err_msg=f"state {i}: pbar")
        if spatial:
            for key in ["h", "q", "q_targ", "n_ap", "n_at"]:
                assert gs[key] == os_[key], f"state {i}: {key} {gs[key]} != {os_[key]}"
            np.testing.assert_array_equal(gs["cnt"], os_["cnt"], err_msg=f"state {i}: cnt")
            np.testing.assert_array_equal(gs["tcnt"], os_["tcnt"], err_msg=f"state {i}: tcnt")
            stale_o = ((os_["ever"] == 1) & (os_["cnt"] == 0)).astype(np.uint8)
            np.testing.assert_array_equal(gs["stale"], stale_o, err_msg=f"state {i}: stale")
    return worst


def sim(W, H, n, seed, scene="sine_checker", noise=0.0, **kw):
    spec = scene if not isinstance(scene, str) else eventsim.SceneSpec(texture=scene, **kw)
    return eventsim.simulate(W, H, n, scene=spec, seed=seed, noise_frac=noise)

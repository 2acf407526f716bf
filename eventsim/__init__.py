"""Seeded contrast-threshold event-camera simulator (synthetic input generator).

This module produces the synthetic event streams that both the FP64 oracle and the
CUDA library consume.  It holds none of FIBAR's arithmetic: it only models a sensor
that emits an ON/OFF event whenever a pixel's log intensity moves by more than the
contrast threshold ``C`` from the level at which it last fired (the event-generation
model of the paper's Sec. 3, Eqs. 1-3).

Record layout (16 bytes, little endian), identical to ``fibar_event_t``::

    uint16 x, uint16 y, int8 p, uint8 pad[3], uint64 t_us

Streams are returned as a contiguous ``torch.int64`` tensor of shape ``(n, 2)``:
word 0 packs ``x | y << 16 | (p & 0xff) << 32``, word 1 is ``t_us``.

Textures (all self-written from their published definitions):

* ``"sine_checker"`` - a sinusoid grating plus a soft-edged checkerboard translated
  at a constant velocity (200 px/s by default).
* ``"perlin"`` - fractal gradient noise (Perlin's improved noise, 2002: quintic fade,
  hashed lattice gradients) that rotates and zooms about the image centre.
* ``"perlin_pan"`` - the same noise panned with piecewise-constant velocities whose
  segment speeds are drawn log-uniformly, giving bursty event rates.

Every random draw comes from numpy's counter-based Philox generator seeded from
``seed``; the per-step sensor model runs in float32 torch ops on ``device``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

EVENT_BYTES = 16
EVENT_NP_DTYPE = np.dtype(
    [("x", "<u2"), ("y", "<u2"), ("p", "i1"), ("pad", "u1", (3,)), ("t", "<u8")]
)
assert EVENT_NP_DTYPE.itemsize == EVENT_BYTES


def pack_events(x, y, p, t_us) -> torch.Tensor:
    """Pack integer tensors into the (n, 2) int64 record layout."""
    x = torch.as_tensor(x).to(torch.int64)
    y = torch.as_tensor(y).to(torch.int64)
    p = torch.as_tensor(p).to(torch.int64)
    t_us = torch.as_tensor(t_us).to(torch.int64)
    w0 = (x & 0xFFFF) | ((y & 0xFFFF) << 16) | ((p & 0xFF) << 32)
    return torch.stack([w0, t_us], dim=1).contiguous()


def unpack_events(ev: torch.Tensor):
    """Inverse of :func:`pack_events`: returns int64 tensors x, y, p (signed), t_us."""
    w0 = ev[:, 0]
    x = w0 & 0xFFFF
    y = (w0 >> 16) & 0xFFFF
    p8 = (w0 >> 32) & 0xFF
    p = torch.where(p8 >= 128, p8 - 256, p8)
    return x, y, p, ev[:, 1]


def to_numpy_records(ev: torch.Tensor) -> np.ndarray:
    """View an (n, 2) int64 tensor as a numpy array of ``EVENT_NP_DTYPE`` records."""
    a = ev.detach().cpu().contiguous().numpy()
    return a.view(EVENT_NP_DTYPE).reshape(-1)


# ----------------------------------------------------------------------------------
# textures (values in [0, 1])
# ----------------------------------------------------------------------------------

_GRAD8 = np.array(
    [[1, 0], [-1, 0], [0, 1], [0, -1], [0.7071067811865476, 0.7071067811865476],
     [-0.7071067811865476, 0.7071067811865476], [0.7071067811865476, -0.7071067811865476],
     [-0.7071067811865476, -0.7071067811865476]], dtype=np.float32)


class _Perlin:
    """2-D gradient noise with a seeded permutation table (Perlin 2002)."""

    def __init__(self, rng: np.random.Generator, device, octaves=4):
        perm = rng.permutation(256).astype(np.int64)
        self.perm = torch.from_numpy(np.concatenate([perm, perm])).to(device)
        self.grad = torch.from_numpy(_GRAD8).to(device)
        self.octaves = octaves

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)

    def _noise(self, u, v):
        fu = torch.floor(u)
        fv = torch.floor(v)
        xi = fu.to(torch.int64) & 255
        yi = fv.to(torch.int64) & 255
        du = u - fu
        dv = v - fv
        perm = self.perm

        def corner(ox, oy):
            h = perm[perm[(xi + ox) & 255] + ((yi + oy) & 255)] & 7
            g = self.grad[h]
            return g[..., 0] * (du - ox) + g[..., 1] * (dv - oy)

        a = self._fade(du)
        b = self._fade(dv)
        n00, n10, n01, n11 = corner(0, 0), corner(1, 0), corner(0, 1), corner(1, 1)
        nx0 = n00 + a * (n10 - n00)
        nx1 = n01 + a * (n11 - n01)
        return nx0 + b * (nx1 - nx0)

    def __call__(self, u, v):
        total = torch.zeros_like(u)
        amp, freq, norm = 1.0, 1.0, 0.0
        for _ in range(self.octaves):
            total = total + amp * self._noise(u * freq, v * freq)
            norm += amp
            amp *= 0.5
            freq *= 2.0
        # gradient noise lies in about [-0.71, 0.71] per octave; map to [0, 1]
        return torch.clamp(0.5 + 0.7 * total / norm, 0.0, 1.0)


@dataclass
class SceneSpec:
    texture: str = "sine_checker"
    speed_px_s: float = 200.0      # translation speed (sine_checker)
    direction_deg: float = 30.0
    period_px: float = 37.0        # sinusoid period
    cell_px: float = 24.0          # checker cell size
    perlin_scale_px: float = 96.0  # lattice spacing of the coarsest octave
    rot_rad_s: float = 0.6         # perlin: rotation rate
    zoom_amp: float = 0.35         # perlin: zoom amplitude (relative)
    zoom_hz: float = 0.25
    pan_rate_lo: float = 1e6       # perlin_pan: events/s range of the bursts
    pan_rate_hi: float = 50e6


class _Scene:
    def __init__(self, spec: SceneSpec, W: int, H: int, rng: np.random.Generator, device):
        self.spec = spec
        self.W, self.H = W, H
        self.device = device
        ys, xs = torch.meshgrid(
            torch.arange(H, dtype=torch.float32, device=device),
            torch.arange(W, dtype=torch.float32, device=device), indexing="ij")
        self.xs = xs.reshape(-1)
        self.ys = ys.reshape(-1)
        self.cx = (W - 1) / 2.0
        self.cy = (H - 1) / 2.0
        self.offset = rng.uniform(0, 1000, size=2)
        if spec.texture in ("perlin", "perlin_pan"):
            self.noise = _Perlin(rng, device)
        if spec.texture == "perlin_pan":
            # piecewise-constant pan: segment durations and speeds from the seed
            nseg = 4096
            self.seg_dur = rng.uniform(0.02, 0.2, size=nseg)
            logr = rng.uniform(math.log(spec.pan_rate_lo), math.log(spec.pan_rate_hi), size=nseg)
            self.seg_rate = np.exp(logr)
            ang = rng.uniform(0, 2 * math.pi, size=nseg)
            self.seg_dir = np.stack([np.cos(ang), np.sin(ang)], axis=1)
            self.seg_t0 = np.concatenate([[0.0], np.cumsum(self.seg_dur)[:-1]])
            self.px_per_event = None  # calibrated lazily

    def pan_position(self, t: float):
        """Integrated pan offset (px) at time t; speed = rate * px_per_event."""
        s = self.spec
        k = int(np.searchsorted(self.seg_t0, t, side="right") - 1)
        k = max(0, min(k, len(self.seg_t0) - 1))
        speeds = self.seg_rate * self.px_per_event
        disp = self.seg_dir * (speeds * self.seg_dur)[:, None]
        base = disp[:k].sum(axis=0)
        return base + self.seg_dir[k] * speeds[k] * (t - self.seg_t0[k])

    def pan_speed(self, t: float) -> float:
        k = int(np.searchsorted(self.seg_t0, t, side="right") - 1)
        k = max(0, min(k, len(self.seg_t0) - 1))
        return float(self.seg_rate[k] * self.px_per_event)

    def texture(self, t: float) -> torch.Tensor:
        s = self.spec
        ox, oy = float(self.offset[0]), float(self.offset[1])
        if s.texture == "sine_checker":
            ang = math.radians(s.direction_deg)
            u = self.xs + (ox + s.speed_px_s * math.cos(ang) * t)
            v = self.ys + (oy + s.speed_px_s * math.sin(ang) * t)
            k = 2.0 * math.pi / s.period_px
            sine = 0.5 + 0.5 * torch.sin(k * u) * torch.sin(k * v)
            c = math.pi / s.cell_px
            chk = 0.5 + 0.5 * torch.tanh(3.0 * torch.sin(c * u) * torch.sin(c * v))
            return 0.45 * sine + 0.55 * chk
        if s.texture == "perlin":
            th = s.rot_rad_s * t
            z = 1.0 + s.zoom_amp * math.sin(2.0 * math.pi * s.zoom_hz * t)
            cs, sn = math.cos(th), math.sin(th)
            dx = self.xs - self.cx
            dy = self.ys - self.cy
            u = (cs * dx - sn * dy) / (z * s.perlin_scale_px) + ox
            v = (sn * dx + cs * dy) / (z * s.perlin_scale_px) + oy
            return self.noise(u, v)
        if s.texture == "perlin_pan":
            px, py = self.pan_position(t)
            u = (self.xs + px) / s.perlin_scale_px + ox
            v = (self.ys + py) / s.perlin_scale_px + oy
            return self.noise(u, v)
        raise ValueError(f"unknown texture {s.texture!r}")

    def log_intensity(self, t: float) -> torch.Tensor:
        return torch.log(0.05 + self.texture(t))


def _make_scene(scene: SceneSpec, W: int, H: int, rng: np.random.Generator, device, C: float) -> _Scene:
    sc = _Scene(scene, W, H, rng, device)
    if scene.texture == "perlin_pan":
        # calibrate events per px of pan motion with a short probe pan along x
        sc.px_per_event = 1.0
        I0 = torch.log(0.05 + sc.noise((sc.xs) / scene.perlin_scale_px + float(sc.offset[0]),
                                       sc.ys / scene.perlin_scale_px + float(sc.offset[1])))
        I1 = torch.log(0.05 + sc.noise((sc.xs + 1.0) / scene.perlin_scale_px + float(sc.offset[0]),
                                       sc.ys / scene.perlin_scale_px + float(sc.offset[1])))
        ev_per_px = float(torch.abs(I1 - I0).sum().item()) / C
        sc.px_per_event = 1.0 / max(ev_per_px, 1.0)
    return sc


def ground_truth(W: int, H: int, *, scene: SceneSpec | str = "sine_checker", seed: int = 0, C: float = 0.2,
                 device: str | torch.device = "cpu"):
    """The scene that ``simulate`` with the same arguments samples, as a function of time:
    returns ``f(t_us) -> (H, W) float32`` log intensity log(0.05 + texture) at t_us."""
    if isinstance(scene, str):
        scene = SceneSpec(texture=scene)
    rng = np.random.Generator(np.random.Philox(seed))
    sc = _make_scene(scene, W, H, rng, torch.device(device), C)
    return lambda t_us: sc.log_intensity(float(t_us) / 1e6).reshape(H, W)


def simulate(W: int, H: int, n_events: int, *, scene: SceneSpec | str = "sine_checker",
             seed: int = 0, C: float = 0.2, noise_frac: float = 0.0,
             device: str | torch.device = "cpu", t0_s: float = 0.0,
             max_dc_per_step: float = 0.6) -> torch.Tensor:
    """Generate exactly ``n_events`` events, sorted by (t_us, pixel, emission order).

    The sensor samples the scene's log intensity at times t_0 < t_1 < ...; after each
    sample, every pixel whose level differs from its reference by at least ``C`` emits
    one event per crossed multiple of ``C`` (sign of the change) with a timestamp
    linearly interpolated between the two samples, and moves its reference by ``C``
    per event.  The sample interval adapts so that the largest per-step change stays
    near ``max_dc_per_step * C``.  ``noise_frac`` of the events are replaced by uniform
    noise (random pixel, random polarity, uniform time over the signal's span).
    """
    if isinstance(scene, str):
        scene = SceneSpec(texture=scene)
    device = torch.device(device)
    rng = np.random.Generator(np.random.Philox(seed))
    sc = _make_scene(scene, W, H, rng, device, C)
    n_noise = int(round(n_events * noise_frac))
    n_signal = n_events - n_noise

    t = t0_s
    I_prev = sc.log_intensity(t)
    ref = I_prev.clone()
    dt = 1e-4
    chunks_t, chunks_pix, chunks_p = [], [], []
    count = 0
    npix = W * H
    steps = 0
    while count < n_signal:
        if scene.texture == "perlin_pan":
            # at most 0.2 px of pan motion per sample: the step size adapts to the
            # intensity change, but a segment's speed can jump at its start
            dt = min(dt, 0.2 / max(sc.pan_speed(t), 1e-3))
        t1 = t + dt
        I = sc.log_intensity(t1)
        d = I - ref
        nc = torch.floor(torch.abs(d) / C)
        hit = nc > 0
        if bool(hit.any()):
            idx = torch.nonzero(hit).squeeze(1)
            ncnt = nc[idx].to(torch.int64)
            sgn = torch.sign(d[idx])
            rep_idx = torch.repeat_interleave(idx, ncnt)
            rep_sgn = torch.repeat_interleave(sgn, ncnt)
            # crossing number m = 1..ncnt for each pixel
            starts = torch.cumsum(ncnt, 0) - ncnt
            m = torch.arange(rep_idx.numel(), device=device) - torch.repeat_interleave(starts, ncnt) + 1
            level = ref[rep_idx] + rep_sgn * m.to(torch.float32) * C
            i0 = I_prev[rep_idx]
            i1 = I[rep_idx]
            frac = torch.clamp((level - i0) / (i1 - i0), 0.0, 1.0)
            tt = t + dt * frac.to(torch.float64)
            t_us = torch.floor(tt * 1e6).to(torch.int64)
            ref[idx] = ref[idx] + sgn * ncnt.to(torch.float32) * C
            chunks_t.append(t_us)
            chunks_pix.append(rep_idx)
            chunks_p.append(rep_sgn.to(torch.int64))
            count += rep_idx.numel()
        maxd = float(torch.abs(I - I_prev).max().item())
        I_prev = I
        t = t1
        steps += 1
        # adapt the sample interval towards max_dc_per_step * C per step
        if maxd > 0:
            dt = min(dt * 1.5, max(dt * 0.25, dt * (max_dc_per_step * C) / maxd))
        else:
            dt *= 1.5
        if steps > 10_000_000:
            raise RuntimeError("simulator did not reach the requested event count")

    t_all = torch.cat(chunks_t)
    pix_all = torch.cat(chunks_pix)
    p_all = torch.cat(chunks_p)
    # order within the signal: (t_us, pixel, emission order)
    key = t_all * npix + pix_all
    order = torch.sort(key, stable=True).indices
    order = order[:n_signal]
    t_all, pix_all, p_all = t_all[order], pix_all[order], p_all[order]

    if n_noise > 0:
        t_lo = int(t_all[0].item()) if n_signal else 0
        t_hi = int(t_all[-1].item()) if n_signal else 1
        nt = rng.integers(t_lo, t_hi + 1, size=n_noise, dtype=np.int64)
        npx = rng.integers(0, npix, size=n_noise, dtype=np.int64)
        npol = rng.integers(0, 2, size=n_noise, dtype=np.int64) * 2 - 1
        t_all = torch.cat([t_all, torch.from_numpy(nt).to(device)])
        pix_all = torch.cat([pix_all, torch.from_numpy(npx).to(device)])
        p_all = torch.cat([p_all, torch.from_numpy(npol).to(device)])
        key = t_all * npix + pix_all
        order = torch.sort(key, stable=True).indices
        t_all, pix_all, p_all = t_all[order], pix_all[order], p_all[order]

    x = pix_all % W
    y = pix_all // W
    return pack_events(x, y, p_all, t_all)


# the workloads the benchmarks and parity tests use --------------------------------

CONFIGS = {
    # 240x180, 1 M events, translating sinusoid+checker at 200 px/s, seed 0, one read-out
    "sine_checker_240x180_1M": dict(W=240, H=180, n_events=1_000_000, scene="sine_checker",
                                   seed=0, noise_frac=0.0),
    # 1280x720, rotating+zooming Perlin noise, 2 % uniform noise events, seed 1
    "perlin_1280x720_200M": dict(W=1280, H=720, n_events=200_000_000, scene="perlin",
                                 seed=1, noise_frac=0.02),
    # 1280x720, bursty pans (1-50 Mev/s segments), seed 2
    "perlin_pan_1280x720_1B": dict(W=1280, H=720, n_events=1_000_000_000, scene="perlin_pan",
                                   seed=2, noise_frac=0.0),
}


def make_config(name: str, n_events: int | None = None, device="cpu", **over) -> torch.Tensor:
    cfg = dict(CONFIGS[name])
    if n_events is not None:
        cfg["n_events"] = n_events
    cfg.update(over)
    return simulate(cfg.pop("W"), cfg.pop("H"), cfg.pop("n_events"), device=device, **cfg)


def random_events(W: int, H: int, n: int, seed: int, *, t_step_us: int = 1,
                  pixels: np.ndarray | None = None, p_on: float = 0.5) -> torch.Tensor:
    """Uniform random events (Philox), optionally restricted to a pixel list.

    Timestamps increase by ``t_step_us`` per event.  Used for small edge-case streams.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    if pixels is None:
        pix = rng.integers(0, W * H, size=n, dtype=np.int64)
    else:
        pix = np.asarray(pixels, dtype=np.int64)[rng.integers(0, len(pixels), size=n)]
    p = np.where(rng.random(n) < p_on, 1, -1).astype(np.int64)
    t = np.arange(n, dtype=np.int64) * t_step_us
    return pack_events(torch.from_numpy(pix % W), torch.from_numpy(pix // W),
                       torch.from_numpy(p), torch.from_numpy(t))


def hot_pixel_events(W: int, H: int, n: int, seed: int, *, hot: list[tuple[int, int]],
                     hot_frac: float = 0.9, t_step_us: int = 1) -> torch.Tensor:
    """A stream dominated by a few flickering ("hot") pixels: each event is, with
    probability ``hot_frac``, on one of the ``hot`` (x, y) pixels (uniformly), else on a
    uniform random pixel; random polarity; time stamps increase by ``t_step_us``.  Hot
    pixels are a common defect of event sensors; here they give one pixel or one tile
    very long event chains."""
    rng = np.random.Generator(np.random.Philox(seed))
    hp = np.asarray([y * W + x for x, y in hot], dtype=np.int64)
    pix = rng.integers(0, W * H, size=n, dtype=np.int64)
    on_hot = rng.random(n) < hot_frac
    pix[on_hot] = hp[rng.integers(0, len(hp), size=int(on_hot.sum()))]
    p = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int64)
    t = np.arange(n, dtype=np.int64) * t_step_us
    return pack_events(torch.from_numpy(pix % W), torch.from_numpy(pix // W),
                       torch.from_numpy(p), torch.from_numpy(t))


# batched serving: many streams of mixed sensors ------------------------------------

SERVING_SENSORS = [(240, 180), (346, 260), (640, 480), (1280, 720)]


def retime(ev: torch.Tensor, seconds: float) -> torch.Tensor:
    """Rescale a stream's time stamps linearly (integer arithmetic, order kept) so that
    it spans [0, seconds]: its mean event rate becomes n / seconds."""
    out = ev.clone()
    if ev.shape[0] == 0:
        return out
    t = ev[:, 1]
    t0 = t[0]
    span = max(int(t[-1].item() - t0.item()), 1)
    out[:, 1] = (t - t0) * int(round(seconds * 1e6)) // span
    return out


def mixed_streams(n_streams: int = 32, seconds: float = 0.2, *, seed: int = 11,
                  sensors=None, rate_lo: float = 0.5e6, rate_hi: float = 20e6,
                  noise_frac: float = 0.02, device="cpu", min_events: int = 1000) -> list[dict]:
    """Seeded streams for batched serving: stream i uses sensor i mod len(sensors) and a
    mean event rate drawn log-uniformly from [rate_lo, rate_hi] events/s; its scene
    alternates between the rotating Perlin texture and the sine+checker; its time stamps
    are rescaled to span `seconds`.
    Returns dicts {W, H, rate, scene, events}."""
    sensors = sensors or SERVING_SENSORS
    rng = np.random.Generator(np.random.Philox(seed))
    scenes = ["perlin", "sine_checker"]
    out = []
    for i in range(n_streams):
        W, H = sensors[i % len(sensors)]
        rate = math.exp(rng.uniform(math.log(rate_lo), math.log(rate_hi)))
        n = max(min_events, int(rate * seconds))
        scene = scenes[i % len(scenes)]
        ev = simulate(W, H, n, scene=scene, seed=seed * 1000 + i, noise_frac=noise_frac, device=device)
        out.append(dict(W=W, H=H, rate=n / seconds, scene=scene, events=retime(ev, seconds)))
    return out


def request_times(n_streams: int, seconds: float, *, rate_hz: float = 100.0, seed: int = 12) -> list[list[int]]:
    """Read-out request times (microseconds) per stream: a Poisson process of `rate_hz`
    on [0, seconds] (exponential gaps), at least one request per stream at the end."""
    rng = np.random.Generator(np.random.Philox(seed))
    end = int(round(seconds * 1e6))
    out = []
    for _ in range(n_streams):
        ts, t = [], 0.0
        while True:
            t += rng.exponential(1e6 / rate_hz)
            if t >= end:
                break
            ts.append(int(t))
        ts.append(end)
        out.append(ts)
    return out


def serving_schedule(streams: list[dict], requests: list[list[int]], tick_us: int = 1000):
    """Replay order for batched serving: per tick [T, T + tick_us), every stream's events
    with time stamps in the tick as one packet (index range lo:hi), then that tick's
    read-out requests.  Returns [(T, [(i, lo, hi), ...], [(i, t_us), ...]), ...]."""
    ends = [int(s["events"][-1, 1]) if s["events"].shape[0] else 0 for s in streams]
    end = max(ends + [max(r) for r in requests if r])
    tcols = [s["events"][:, 1].cpu().numpy() for s in streams]
    reqs = [np.asarray(r, dtype=np.int64) for r in requests]
    out = []
    for T in range(0, end + 1, tick_us):
        pushes, reads = [], []
        for i, t in enumerate(tcols):
            lo, hi = np.searchsorted(t, [T, T + tick_us], side="left")
            if hi > lo:
                pushes.append((i, int(lo), int(hi)))
        for i, r in enumerate(reqs):
            a, b = np.searchsorted(r, [T, T + tick_us], side="left")
            reads.extend((i, int(x)) for x in r[a:b])
        out.append((T, pushes, reads))
    return out


# threshold calibration recordings ---------------------------------------------------

def threshold_recording(W: int, H: int, *, periods: int = 20, amplitude: float = 1.0,
                        period_s: float = 1.0, c_mean: float = 0.2, spread: float = 0.15,
                        imbalance: float = 0.25, steps_per_half: int = 64, seed: int = 5):
    """A sensor with per-pixel ON / OFF thresholds watching a spatially uniform log
    brightness that follows a triangle wave (the setup of the paper's appendix on
    relative thresholds: an exponentially ramped illumination gives a linear triangle
    in log brightness).  Thresholds: c_mean * exp(N(0, spread) +- N(0, imbalance) / 2)
    for ON / OFF.  Each pixel starts at a random level within its thresholds; an event
    fires whenever the brightness moves a threshold away from the pixel's reference,
    stamped at the linear crossing time.  Returns dict(events, c_on, c_off) with (H, W)
    float64 threshold arrays."""
    rng = np.random.Generator(np.random.Philox(seed))
    n = W * H
    base = rng.normal(0.0, spread, n)
    imb = rng.normal(0.0, imbalance, n)
    c_on = c_mean * np.exp(base + imb / 2)
    c_off = c_mean * np.exp(base - imb / 2)
    # step must move the brightness less than any threshold: at most one event per step
    dl = amplitude / steps_per_half
    if dl >= min(c_on.min(), c_off.min()):
        raise ValueError("steps_per_half too small for the thresholds")
    ref = rng.uniform(-c_off, c_on)  # level of the last event relative to the start
    dt_us = period_s / 2 / steps_per_half * 1e6
    level = 0.0
    ts, pix, pol = [], [], []
    idx = np.arange(n)
    nsteps = 2 * steps_per_half * periods
    for st in range(nsteps):
        up = (st // steps_per_half) % 2 == 0
        new = level + (dl if up else -dl)
        if up:
            hit = new - ref >= c_on
            cross = ref + c_on
        else:
            hit = ref - new >= c_off
            cross = ref - c_off
        k = idx[hit]
        if k.size:
            frac = (cross[k] - level) / (new - level)
            ts.append(np.floor((st + frac) * dt_us).astype(np.int64))
            pix.append(k)
            pol.append(np.full(k.size, 1 if up else -1, dtype=np.int64))
            ref[k] = cross[k]
        level = new
    t = np.concatenate(ts) if ts else np.zeros(0, np.int64)
    p_ = np.concatenate(pix) if pix else np.zeros(0, np.int64)
    s_ = np.concatenate(pol) if pol else np.zeros(0, np.int64)
    order = np.lexsort((p_, t))
    t, p_, s_ = t[order], p_[order], s_[order]
    ev = pack_events(torch.from_numpy(p_ % W), torch.from_numpy(p_ // W), torch.from_numpy(s_), torch.from_numpy(t))
    return dict(events=ev, c_on=c_on.reshape(H, W), c_off=c_off.reshape(H, W))

"""Learned stale-pixel fill: training data, training loop and evaluation.

The network and its kernels are in the library (``csrc/k_fill.cu``; C ABI
``fibar_fill_*``); this module only marshals data for them.  A training frame is one
read-out of a FIBAR stream: the network's inputs (L and the activity age, from
``fibar_fill_features``), the stale mask, and the target: the simulator's log
intensity I at the read-out time in L units, T = (I - b) / a with (a, b) the least-squares
fit I ~ a L + b over the frame's active pixels (had an event, still queued).  L is a
high-passed log brightness (Eqs. 9-10 remove its DC), so I has to be mapped into its
units before a fill can be scored against it.  The loss is the mean squared error over
stale pixels; the Gaussian fill of the S2 read-out is scored with the same metric.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import binding as B

CROP = 24      # training crop side (the kernel's fixed crop)
MARGIN = 3     # pixels at a crop border without a full receptive field


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in), fan_in = 9 x input channels), zero
    biases, the last layer scaled by 0.1; FP32, in the library's parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for cout, cin in [(16, 2), (16, 16), (1, 16)]:
        lim = math.sqrt(6.0 / (9 * cin))
        w = rng.uniform(-lim, lim, size=cout * cin * 9)
        if cout == 1:
            w *= 0.1
        parts += [w, np.zeros(cout)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == B.FIBAR_FILL_NPARAMS
    return theta


def affine_target(L: torch.Tensor, I: torch.Tensor, active: torch.Tensor) -> torch.Tensor:
    """T = (I - b) / a with a, b the least-squares fit I ~ a L + b over `active` pixels
    (sums in float64)."""
    l = L[active].double()
    i = I[active].double()
    n = l.numel()
    sl, si = l.sum(), i.sum()
    sll, sli = (l * l).sum(), (l * i).sum()
    a = (n * sli - sl * si) / (n * sll - sl * sl)
    b = (si - a * sl) / n
    return ((I.double() - b) / a).float()


class Frames:
    """Training or evaluation frames on the device: X [F, 2, H, W], T [F, H, W],
    stale [F, H, W] (uint8), gauss [F, H, W] (the S2 read-out image)."""

    def __init__(self, X, T, stale, gauss):
        self.X, self.T, self.stale, self.gauss = X, T, stale, gauss

    @property
    def n(self):
        return self.X.shape[0]

    @staticmethod
    def concat(parts):
        return Frames(*(torch.cat([getattr(p, k) for p in parts]) for k in ("X", "T", "stale", "gauss")))


def collect_frames(W: int, H: int, n_events: int, *, seed: int, scene: str = "perlin", noise: float = 0.02,
                   read_every: int = 1_000_000, skip: int = 2, packet: int = 65_536, C: float = 0.2) -> Frames:
    """Run a seeded simulator stream through an S2 handle and keep one frame per read-out
    (after `skip` read-outs of queue start-up)."""
    import eventsim
    ev = eventsim.simulate(W, H, n_events, scene=scene, seed=seed, noise_frac=noise, device="cuda")
    truth = eventsim.ground_truth(W, H, scene=scene, seed=seed, C=C, device="cuda")
    f = B.Fibar(W, H, c_on=C, c_off=C, spatial_filter=1, blur_mode=1)
    Xs, Ts, Ss, Gs = [], [], [], []
    pos, r = 0, 0
    try:
        while pos + read_every <= n_events:
            for lo in range(pos, pos + read_every, packet):
                f.push(ev[lo:min(lo + packet, pos + read_every)])
            t_read = int(ev[pos + read_every - 1, 1].item())
            img = f.readout(t_read)
            pos += read_every
            r += 1
            if r <= skip:
                continue
            x, st = f.fill_features()
            I = truth(t_read)
            active = (x[1] < 2.0) & (st == 0)   # had an event (age below the cap of 4) and still queued
            Xs.append(x)
            Ts.append(affine_target(x[0], I, active))
            Ss.append(st)
            Gs.append(img.clone())
    finally:
        f.close()
    return Frames(torch.stack(Xs), torch.stack(Ts), torch.stack(Ss), torch.stack(Gs))


def sample_crops(fr: Frames, n: int, gen: torch.Generator) -> torch.Tensor:
    """n random crops (frame, y0, x0) inside the frames, as an int32 CUDA tensor [n, 3]."""
    F, _, H, W = fr.X.shape
    f = torch.randint(0, F, (n,), generator=gen)
    y = torch.randint(0, H - CROP + 1, (n,), generator=gen)
    x = torch.randint(0, W - CROP + 1, (n,), generator=gen)
    return torch.stack([f, y, x], 1).to(torch.int32).cuda()


class Trainer:
    """Adam on FP32 master weights through ``fibar_fill_train_step``."""

    def __init__(self, theta0: np.ndarray, lr: float = 2e-3):
        self.theta = torch.from_numpy(np.asarray(theta0, dtype=np.float32).copy()).cuda()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.acc = torch.zeros(3, dtype=torch.float64, device="cuda")
        self.lr = lr
        self.t = 0

    def step(self, fr: Frames, crops: torch.Tensor, lr: float | None = None) -> None:
        """One Adam step (lr = 0: gradient only, in self.grad)."""
        self.t += 1
        lr = self.lr if lr is None else lr
        F, _, H, W = fr.X.shape
        s = torch.cuda.current_stream().cuda_stream
        M = fr.stale
        rc = B.fibar_fill_train_step(fr.X.data_ptr(), fr.T.data_ptr(), M.data_ptr(), W, H, F, crops.data_ptr(),
                                     crops.shape[0], self.theta.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                     self.grad.data_ptr(), self.t, float(lr), self.acc.data_ptr(), s)
        if rc != 0:
            raise B.FibarError(rc, "fibar_fill_train_step failed")

    def loss(self) -> float:
        a = self.acc.cpu().numpy()
        return float(a[0] / max(a[1], 1.0))

    def params(self) -> np.ndarray:
        return self.theta.cpu().numpy()


def train(fr: Frames, steps: int, *, batch: int = 512, lr: float = 2e-3, seed: int = 0, theta0=None,
          log_every: int = 0):
    """Train from theta0 (default: init_params(seed)); returns (theta, seconds, loss history)."""
    tr = Trainer(init_params(seed) if theta0 is None else theta0, lr)
    gen = torch.Generator().manual_seed(seed)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        # cosine decay to a tenth of the initial rate
        lr_i = lr * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * i / max(steps - 1, 1))))
        tr.step(fr, sample_crops(fr, batch, gen), lr_i)
        if log_every and (i % log_every == 0 or i == steps - 1):
            hist.append((i, tr.loss()))
    torch.cuda.synchronize()
    return tr.params(), time.perf_counter() - t0, hist


def evaluate(theta: np.ndarray, fr: Frames) -> dict:
    """RMSE against the target over the stale pixels at least MARGIN from the border:
    the learned fill, the Gaussian fill (S2 image) and no fill (L itself)."""
    se = {"learned": 0.0, "gaussian": 0.0, "none": 0.0}
    n = 0
    for i in range(fr.n):
        out = B.fill_forward(theta, fr.X[i].contiguous(), fr.stale[i].contiguous())
        m = fr.stale[i].bool().clone()
        m[:MARGIN, :] = False
        m[-MARGIN:, :] = False
        m[:, :MARGIN] = False
        m[:, -MARGIN:] = False
        t = fr.T[i][m].double()
        se["learned"] += float(((out[m].double() - t) ** 2).sum())
        se["gaussian"] += float(((fr.gauss[i][m].double() - t) ** 2).sum())
        se["none"] += float(((fr.X[i, 0][m].double() - t) ** 2).sum())
        n += int(m.sum())
    return {k: math.sqrt(v / max(n, 1)) for k, v in se.items()} | {"pixels": n}

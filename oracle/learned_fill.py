"""Learned stale-pixel fill: plain FP64 oracle - TEST INFRASTRUCTURE ONLY.

FIBAR fills a pixel that went stale with an isotropic 3x3 Gaussian of its neighbours
(Sec. 4.2).  The paper's limitations section criticises exactly that (the blur ignores
the gradient's magnitude and direction) and defers "more sophisticated algorithms" to
GPUs.  This module defines one such algorithm and is the reference the CUDA kernels are
checked against; nothing in the product path imports it.

Fill network (the read-out's masked fill, S2 mask):
  input   x[0] = L                  FIBAR's filter output (Eq. 10), unblurred
          x[1] = age = min(A_MAX, (k - last) / q)
                 k the events applied, last the global index of the pixel's last event,
                 q the queue length (the window of Sec. 4.2 is [k - q, k)); a pixel is
                 stale exactly when age > 1; a pixel without events has age = A_MAX
  conv1   z1 = b1 + W1 * bf16(x)  (2 -> 16 channels, 3x3, zero padding), a1 = relu(z1)
  conv2   z2 = b2 + W2 * bf16(a1)  (16 -> 16), a2 = relu(z2)
  conv3   y  = b3 + W3 * bf16(a2)  (16 -> 1)
  output  out = y where the pixel is stale (had an event, none queued), L elsewhere
"*" is a cross-correlation: (W * x)[c, i, j] = sum over ci, dy, dx in {0,1,2} of
W[c, ci, dy, dx] x[ci, i + dy - 1, j + dx - 1], zero outside the image.  All three layers
are tensor-core contractions with BF16 operands and FP32 accumulation: the weights (W1,
W2, W3) and each layer's input (x, a1, a2) are rounded to bfloat16, biases stay FP32;
everything else is exact here (FP64).  Outside the stale pixels the output is L itself
(not its BF16 rounding).

Training target (a reading: L is a high-passed log brightness, Eqs. 9-10 remove its DC,
so it cannot be compared with the simulator's log intensity I directly): per frame, the
affine map I ~ a L + b fitted by least squares over the active pixels (had an event and
still queued) converts I into L units, T = (I - b) / a; the loss is the mean squared
error of y against T over the stale pixels (of the interior of each training crop, where
the 7x7 receptive field lies inside the crop).  Optimiser: Adam (Kingma & Ba, 2015).
"""
from __future__ import annotations

import numpy as np

A_MAX = 4.0      # cap of the age feature (pixels without events sit at the cap)
C_IN, C_HID = 2, 16
MARGIN = 3       # receptive-field margin of three 3x3 layers


# -- bfloat16 rounding from its definition: float32 with the low 16 bits rounded off
#    (round to nearest, ties to even); used for the weights and for a1 -------------

def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# -- parameters -----------------------------------------------------------------

SHAPES = {"W1": (C_HID, C_IN, 3, 3), "b1": (C_HID,), "W2": (C_HID, C_HID, 3, 3), "b2": (C_HID,),
          "W3": (1, C_HID, 3, 3), "b3": (1,)}
ORDER = ["W1", "b1", "W2", "b2", "W3", "b3"]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES.values())


def unflatten(theta) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = theta[o:o + n].reshape(SHAPES[k])
        o += n
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1) for k in ORDER])


# -- features and target ---------------------------------------------------------

def age_feature(k: int, q: int, last: np.ndarray) -> np.ndarray:
    """min(A_MAX, (k - last) / q); A_MAX where last is the 'no event' marker 2^64 - 1."""
    last = np.asarray(last, dtype=np.uint64)
    never = last == np.uint64(0xFFFFFFFFFFFFFFFF)
    gap = (np.uint64(k) - np.where(never, np.uint64(0), last)).astype(np.float64)
    a = np.minimum(A_MAX, gap / float(max(q, 1)))
    return np.where(never, A_MAX, a)


def stale_mask(h: int, last: np.ndarray) -> np.ndarray:
    """Had an event and has none in the window [h, k) (the S2 read-out's mask)."""
    last = np.asarray(last, dtype=np.uint64)
    return (last != np.uint64(0xFFFFFFFFFFFFFFFF)) & (last < np.uint64(h))


def affine_target(L: np.ndarray, I: np.ndarray, active: np.ndarray):
    """Least-squares a, b of I ~ a L + b over the active pixels; returns (T, a, b) with
    T = (I - b) / a the ground truth in L units."""
    l = np.asarray(L, dtype=np.float64)[active]
    i = np.asarray(I, dtype=np.float64)[active]
    n = l.size
    sl, si = l.sum(), i.sum()
    sll, sli = (l * l).sum(), (l * i).sum()
    a = (n * sli - sl * si) / (n * sll - sl * sl)
    b = (si - a * sl) / n
    return (np.asarray(I, dtype=np.float64) - b) / a, a, b


# -- the network ----------------------------------------------------------------

def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [Cin, H, Wd], W [Cout, Cin, 3, 3], b [Cout] -> [Cout, H, Wd]: the cross-
    correlation with zero padding, as nine shifted multiply-adds."""
    cin, H, Wd = x.shape
    xp = np.zeros((cin, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.broadcast_to(np.asarray(b, dtype=np.float64)[:, None, None], (W.shape[0], H, Wd)).copy()
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,chw->ohw", W[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + Wd])
    return out


def forward(theta, x: np.ndarray, quantize: bool = True) -> dict:
    """Forward pass on one image x [2, H, W]; returns every intermediate."""
    p = unflatten(theta)
    q = bf16 if quantize else (lambda v: np.asarray(v, dtype=np.float64))
    W1, W2, W3 = q(p["W1"]), q(p["W2"]), q(p["W3"])
    xq = q(x)
    z1 = conv3x3(xq, W1, p["b1"])
    a1 = np.maximum(z1, 0.0)
    a1q = q(a1)
    z2 = conv3x3(a1q, W2, p["b2"])
    a2 = np.maximum(z2, 0.0)
    a2q = q(a2)
    y = conv3x3(a2q, W3, p["b3"])[0]
    return dict(W1=W1, W2=W2, W3=W3, xq=xq, z1=z1, a1=a1, a1q=a1q, z2=z2, a2=a2, a2q=a2q, y=y)


def fill_image(theta, L: np.ndarray, age: np.ndarray, stale: np.ndarray) -> np.ndarray:
    """The read-out image: the network's output at stale pixels, L elsewhere."""
    x = np.stack([np.asarray(L, dtype=np.float64), np.asarray(age, dtype=np.float64)])
    y = forward(theta, x)["y"]
    return np.where(stale, y, L)


def conv3x3_backward(x: np.ndarray, W: np.ndarray, g: np.ndarray):
    """Gradients of sum(g * conv3x3(x, W, b)) w.r.t. x, W and b."""
    cin, H, Wd = x.shape
    xp = np.zeros((cin, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W, dtype=np.float64)
    for dy in range(3):
        for dx in range(3):
            dW[:, :, dy, dx] = np.einsum("ohw,chw->oc", g, xp[:, dy:dy + H, dx:dx + Wd])
            dxp[:, dy:dy + H, dx:dx + Wd] += np.einsum("oc,ohw->chw", W[:, :, dy, dx], g)
    return dxp[:, 1:-1, 1:-1], dW, g.sum(axis=(1, 2))


def loss_and_grad(theta, xs, targets, masks, quantize: bool = True):
    """Mean squared error over the masked pixels of a batch of crops and its gradient
    with respect to theta (rounding steps treated as the identity: the gradient is
    evaluated at the rounded values).  xs [B, 2, S, S], targets / masks [B, S, S]."""
    n = float(sum(int(m.sum()) for m in masks))
    grads = {k: np.zeros(SHAPES[k]) for k in ORDER}
    loss = 0.0
    for x, t, m in zip(xs, targets, masks):
        f = forward(theta, x, quantize)
        r = np.where(m, f["y"] - t, 0.0)
        loss += float((r * r).sum()) / n
        gy = (2.0 / n) * r
        da2, grads_W3, gb3 = conv3x3_backward(f["a2q"], f["W3"], gy[None])
        grads["W3"] += grads_W3
        grads["b3"] += gb3
        dz2 = da2 * (f["z2"] > 0)
        da1, gW2, gb2 = conv3x3_backward(f["a1q"], f["W2"], dz2)
        grads["W2"] += gW2
        grads["b2"] += gb2
        dz1 = da1 * (f["z1"] > 0)
        _, gW1, gb1 = conv3x3_backward(f["xq"], f["W1"], dz1)
        grads["W1"] += gW1
        grads["b1"] += gb1
    return loss, flatten(grads)


def adam_step(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step number t >= 1); returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v

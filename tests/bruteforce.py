"""Independent brute-force restatement of FIBAR's stale-pixel detector (test helper).

Written separately from the C oracle to pin it: instead of incremental per-pixel and
per-tile counters, every quantity is recomputed from scratch from the event window at
every step (O(q) per step), so it only suits tiny sensors and short streams.

Paper passages: Sec. 4.2 steps 1-3 (push, pop while longer than q_targ, a pixel whose
last queued event leaves becomes inactive), Eq. 19 (fill ratio over 2x2 tiles, A = 4)
and Eq. 20 (q_targ update, integer form, bounded below by q_min and above by W*H).
"""
from __future__ import annotations


def tile_of(pix: int, W: int) -> tuple[int, int]:
    x, y = pix % W, pix // W
    return (x // 2, y // 2)


def detector_trace(W: int, H: int, pixels, *, fill_num=1, fill_den=2, q_min=None,
                   q_init=None):
    """Run the detector on a pixel sequence; return per-step window data.

    Returns a dict with lists ``h`` (window start after the pops of step k),
    ``q_targ`` (target for step k+1), ``n_ap``, ``n_at`` and ``stale`` (list of
    (k, pixel) in pop order).
    """
    npix = W * H
    if q_min is None:
        q_min = max(1, -(-npix // 1024))
    if q_init is None:
        q_init = q_min
    q_max = npix
    seq = list(pixels)
    h = 0
    q_targ = q_init
    out = dict(h=[], q_targ=[], n_ap=[], n_at=[], stale=[])
    for k in range(len(seq)):
        # window after the push is seq[h..k]; pop from the front while too long
        while (k - h + 1) > q_targ:
            j = h
            h += 1
            # the popped pixel is inactive iff none of its events remains queued
            if seq[j] not in seq[h:k + 1]:
                out["stale"].append((k, seq[j]))
        win = seq[h:k + 1]
        q = len(win)
        n_ap = len(set(win))
        n_at = len({tile_of(p, W) for p in win})
        # Eq. 20 with r_k = n_ap / (4 n_at) and r_fill = fill_num / fill_den
        qt = (q * fill_num * 4 * n_at) // (fill_den * n_ap)
        q_targ = min(max(qt, q_min), q_max)
        out["h"].append(h)
        out["q_targ"].append(q_targ)
        out["n_ap"].append(n_ap)
        out["n_at"].append(n_at)
    return out

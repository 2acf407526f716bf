"""ctypes wrapper around the FP64 oracle (``fibar_oracle.c``) - test infrastructure.

``build()`` compiles the C source with the host gcc into ``oracle/libfibar_ref.so``
(in-tree, git-ignored).  :class:`Oracle` mirrors the library's create / push /
readout / state calls with FP64 outputs and an optional per-event trace.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fibar_oracle.c")
_LIB = os.path.join(_HERE, "libfibar_ref.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class RefEvent(C.Structure):
    _fields_ = [("x", C.c_uint16), ("y", C.c_uint16), ("p", C.c_int8),
                ("pad", C.c_uint8 * 3), ("t_us", C.c_uint64)]


class RefParams(C.Structure):
    _fields_ = [("t_cut", C.c_double), ("fill_num", C.c_uint32), ("fill_den", C.c_uint32),
                ("q_min", C.c_uint32), ("q_init", C.c_uint32), ("c_on", C.c_float),
                ("c_off", C.c_float), ("spatial_filter", C.c_int32),
                ("blur_mode", C.c_int32), ("chain_policy", C.c_int32)]


class RefTrace(C.Structure):
    _fields_ = [("cap", C.c_uint64), ("h", C.POINTER(C.c_uint64)),
                ("q_targ", C.POINTER(C.c_uint64)), ("n_ap", C.POINTER(C.c_uint64)),
                ("n_at", C.POINTER(C.c_uint64)), ("stale_cap", C.c_uint64),
                ("stale_k", C.POINTER(C.c_uint64)), ("stale_pix", C.POINTER(C.c_uint32)),
                ("n_stale", C.c_uint64), ("k0", C.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            vp = C.c_void_p
            lib.fibar_ref_create.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(RefParams), C.POINTER(vp)]
            lib.fibar_ref_create.restype = C.c_int
            lib.fibar_ref_destroy.argtypes = [vp]
            lib.fibar_ref_destroy.restype = None
            lib.fibar_ref_push_events.argtypes = [vp, vp, C.c_uint64]
            lib.fibar_ref_push_events.restype = C.c_int
            lib.fibar_ref_readout.argtypes = [vp, C.c_uint64, vp]
            lib.fibar_ref_readout.restype = C.c_int
            lib.fibar_ref_flush.argtypes = [vp]
            lib.fibar_ref_flush.restype = C.c_int
            lib.fibar_ref_state.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            lib.fibar_ref_state.restype = C.c_int
            lib.fibar_ref_set_trace.argtypes = [vp, C.POINTER(RefTrace)]
            lib.fibar_ref_set_trace.restype = None
            lib.fibar_ref_coefficients.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.fibar_ref_coefficients.restype = None
            lib.fibar_ref_info.argtypes = [vp, vp, vp]
            lib.fibar_ref_info.restype = None
            lib.fibar_ref_blur_image.argtypes = [C.c_uint32, C.c_uint32, vp, vp]
            lib.fibar_ref_blur_image.restype = None
            lib.fibar_ref_set_gain.argtypes = [vp, vp]
            lib.fibar_ref_set_gain.restype = C.c_int
            lib.fibar_ref_relative_thresholds.argtypes = [C.c_uint32, C.c_uint32, vp, C.c_uint64, vp, vp, vp]
            lib.fibar_ref_relative_thresholds.restype = C.c_int
            _lib = lib
    return _lib


def coefficients(t_cut: float):
    """(alpha, beta) of Eqs. 17-18 as the oracle computes them."""
    lib = _load()
    a, b = C.c_double(), C.c_double()
    lib.fibar_ref_coefficients(float(t_cut), C.byref(a), C.byref(b))
    return a.value, b.value


def blur_image(img: np.ndarray) -> np.ndarray:
    """The oracle's border-renormalised 3x3 binomial blur of a whole (H, W) image."""
    lib = _load()
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    out = np.empty_like(img)
    lib.fibar_ref_blur_image(W, H, img.ctypes.data, out.ctypes.data)
    return out


def relative_thresholds(W: int, H: int, ev):
    """Relative contrast thresholds (C'_on, C'_off, C') of every pixel from a calibration
    recording, as (H, W) float64 arrays (NaN where undefined)."""
    lib = _load()
    rec = _as_records(ev)
    n = W * H
    out = [np.empty(n, np.float64) for _ in range(3)]
    rc = lib.fibar_ref_relative_thresholds(W, H, rec.ctypes.data, rec.shape[0],
                                           *[o.ctypes.data for o in out])
    if rc != 0:
        raise ValueError(f"fibar_ref_relative_thresholds failed: {rc}")
    return tuple(o.reshape(H, W) for o in out)


def default_params(**over) -> dict:
    p = dict(t_cut=40.0, fill_num=1, fill_den=2, q_min=0, q_init=0, c_on=1.0, c_off=1.0,
             spatial_filter=1, blur_mode=0, chain_policy=0)
    p.update(over)
    return p


def _as_records(ev) -> np.ndarray:
    """Accept a torch (n,2) int64 tensor, a numpy int64 (n,2) array or a record array."""
    try:
        import torch
        if isinstance(ev, torch.Tensor):
            ev = ev.detach().cpu().contiguous().numpy()
    except ImportError:  # pragma: no cover
        pass
    ev = np.ascontiguousarray(ev)
    if ev.dtype == np.int64 and ev.ndim == 2 and ev.shape[1] == 2:
        return ev
    if ev.dtype.itemsize == 16:
        return ev.view(np.int64).reshape(-1, 2)
    raise TypeError("events must be packed 16-byte records")


class Oracle:
    """One FIBAR stream in the FP64 oracle."""

    def __init__(self, W: int, H: int, **params):
        self.lib = _load()
        self.W, self.H = int(W), int(H)
        p = default_params(**params)
        self._p = RefParams(**p)
        h = C.c_void_p()
        rc = self.lib.fibar_ref_create(self.W, self.H, C.byref(self._p), C.byref(h))
        if rc != 0:
            raise ValueError(f"fibar_ref_create failed: {rc}")
        self.h = h
        self._trace = None
        ab = (C.c_double * 2)()
        qb = (C.c_uint64 * 3)()
        self.lib.fibar_ref_info(self.h, ab, qb)
        self.alpha, self.beta = ab[0], ab[1]
        self.q_min, self.q_max, self.q_init = qb[0], qb[1], qb[2]

    def close(self):
        if self.h:
            self.lib.fibar_ref_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gain(self, gain) -> None:
        """Sec. 5.2 correction: per-pixel factor on Eq. 6 (None removes it)."""
        if gain is None:
            self.lib.fibar_ref_set_gain(self.h, None)
            return
        g = np.ascontiguousarray(np.asarray(gain, dtype=np.float64).reshape(-1))
        if g.size != self.W * self.H:
            raise ValueError("one gain per pixel")
        if self.lib.fibar_ref_set_gain(self.h, g.ctypes.data) != 0:
            raise MemoryError("fibar_ref_set_gain")

    def push(self, ev) -> None:
        rec = _as_records(ev)
        rc = self.lib.fibar_ref_push_events(self.h, rec.ctypes.data, rec.shape[0])
        if rc != 0:
            raise RuntimeError(f"push failed: {rc}")

    def readout(self, t_us: int) -> np.ndarray:
        out = np.empty(self.W * self.H, dtype=np.float64)
        rc = self.lib.fibar_ref_readout(self.h, int(t_us), out.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"readout failed: {rc}")
        return out.reshape(self.H, self.W)

    def readout_rc(self, t_us: int) -> int:
        out = np.empty(self.W * self.H, dtype=np.float64)
        return self.lib.fibar_ref_readout(self.h, int(t_us), out.ctypes.data)

    def flush(self) -> None:
        self.lib.fibar_ref_flush(self.h)

    def state(self) -> dict:
        n = self.W * self.H
        ntiles = ((self.W + 1) // 2) * ((self.H + 1) // 2)
        pbar = np.empty(n, np.float64)
        L = np.empty(n, np.float64)
        cnt = np.empty(n, np.uint32)
        tcnt = np.empty(ntiles, np.uint8)
        ever = np.empty(n, np.uint8)
        last = np.empty(n, np.uint64)
        sc = np.empty(8, np.uint64)
        self.lib.fibar_ref_state(self.h, pbar.ctypes.data, L.ctypes.data, cnt.ctypes.data,
                                 tcnt.ctypes.data, ever.ctypes.data, last.ctypes.data,
                                 sc.ctypes.data)
        keys = ["k", "h", "q", "q_targ", "n_ap", "n_at", "dropped", "pending"]
        d = {k: int(v) for k, v in zip(keys, sc)}
        d.update(pbar=pbar, L=L, cnt=cnt, tcnt=tcnt, ever=ever, last=last)
        return d

    def start_trace(self, cap: int, stale_cap: int | None = None) -> None:
        """Record per-event h, q_targ, N_ap, N_at and the ordered stale list."""
        stale_cap = cap if stale_cap is None else stale_cap
        self._bufs = dict(h=np.zeros(cap, np.uint64), q_targ=np.zeros(cap, np.uint64),
                          n_ap=np.zeros(cap, np.uint64), n_at=np.zeros(cap, np.uint64),
                          stale_k=np.zeros(stale_cap, np.uint64),
                          stale_pix=np.zeros(stale_cap, np.uint32))
        b = self._bufs
        u64p = C.POINTER(C.c_uint64)
        tr = RefTrace(cap=cap, h=b["h"].ctypes.data_as(u64p), q_targ=b["q_targ"].ctypes.data_as(u64p),
                      n_ap=b["n_ap"].ctypes.data_as(u64p), n_at=b["n_at"].ctypes.data_as(u64p),
                      stale_cap=stale_cap, stale_k=b["stale_k"].ctypes.data_as(u64p),
                      stale_pix=b["stale_pix"].ctypes.data_as(C.POINTER(C.c_uint32)),
                      n_stale=0, k0=0)
        self._trace = tr
        self.lib.fibar_ref_set_trace(self.h, C.byref(tr))

    def trace(self) -> dict:
        tr = self._trace
        n = min(int(self.state()["k"]) - int(tr.k0), int(tr.cap))
        ns = min(int(tr.n_stale), int(tr.stale_cap))
        b = self._bufs
        return dict(k0=int(tr.k0), h=b["h"][:n].copy(), q_targ=b["q_targ"][:n].copy(),
                    n_ap=b["n_ap"][:n].copy(), n_at=b["n_at"][:n].copy(),
                    stale_k=b["stale_k"][:ns].copy(), stale_pix=b["stale_pix"][:ns].copy(),
                    n_stale=int(tr.n_stale))

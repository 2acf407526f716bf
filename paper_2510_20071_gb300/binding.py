"""ctypes binding of ``libfibar.so`` (the C ABI of ``include/fibar.h``).

The module-level ``fibar_*`` functions have the C names and signatures.  :class:`Fibar`
is a convenience wrapper that takes torch tensors (for device memory and streams
only) and raises :class:`FibarError` on any non-zero status.
"""
from __future__ import annotations

import array
import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

FIBAR_OK = 0
FIBAR_EINVAL = -1
FIBAR_ENOMEM = -2
FIBAR_EORDER = -3
FIBAR_ECUDA = -4
FIBAR_ETIMEOUT = -5

EXPORTED = ["fibar_default_params", "fibar_create", "fibar_push_events", "fibar_readout",
            "fibar_flush", "fibar_debug_state", "fibar_stats", "fibar_set_timing",
            "fibar_stage_times", "fibar_last_error", "fibar_destroy", "fibar_queue_counts_noalloc",
            "fibar_readout_batch", "fibar_memory_bytes", "fibar_relative_thresholds",
            "fibar_set_pixel_gain", "fibar_debug_wait_timeout", "fibar_push_events_many",
            "fibar_fill_set_weights", "fibar_fill_features", "fibar_fill_forward", "fibar_fill_train_step",
            "fibar_readout_host_async", "fibar_wait", "fibar_set_grid_share", "fibar_push_batch",
            "fibar_group_create", "fibar_group_readout", "fibar_group_latency", "fibar_group_stats",
            "fibar_group_last_error", "fibar_group_destroy", "fibar_group_join"]

FIBAR_FILL_NPARAMS = 2769

STAGES = ["decode", "sort", "walk", "det_counts", "det_pass1", "det_pass2", "det_fix", "s1_blur",
          "readout", "commit"]


class FibarError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fibar error {code}: {msg}")
        self.code = code


class FibarParams(C.Structure):
    _fields_ = [("t_cut", C.c_double), ("fill_num", C.c_uint32), ("fill_den", C.c_uint32),
                ("q_min", C.c_uint32), ("q_init", C.c_uint32), ("c_on", C.c_float),
                ("c_off", C.c_float), ("spatial_filter", C.c_int32), ("blur_mode", C.c_int32),
                ("chain_policy", C.c_int32), ("max_pending", C.c_uint32)]


class FibarStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ["events_pushed", "events_applied", "events_dropped",
                                          "events_pending", "readouts", "q", "q_targ", "n_ap",
                                          "n_at", "detector_fixups", "kernel_launches",
                                          "detector_unmerged", "detector_pass2_steps",
                                          "detector_fix_steps", "s1_blurs", "detector_big_pops",
                                          "detector_ring_misses", "detector_recenters",
                                          "iir_walk_pieces", "iir_scan_pieces"]]


class FibarGroupStats(C.Structure):
    _fields_ = [("members", C.c_uint64), ("graph_launches", C.c_uint64), ("builds", C.c_uint64),
                ("graph_kernels", C.c_uint64), ("programmatic_edges", C.c_int32)]


class FibarStageTimes(C.Structure):
    _fields_ = [("ms", C.c_double * 10), ("calls", C.c_uint64)]


class FibarStateView(C.Structure):
    _fields_ = [("pbar", C.c_void_p), ("L", C.c_void_p), ("cnt", C.c_void_p), ("tcnt", C.c_void_p),
                ("stale", C.c_void_p), ("last_idx", C.c_void_p), ("k", C.c_uint64), ("h", C.c_uint64),
                ("q", C.c_uint64), ("q_targ", C.c_uint64), ("n_ap", C.c_uint64), ("n_at", C.c_uint64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libfibar.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise FibarError(FIBAR_ECUDA, f"CUDA library not built: {_build.LIB}")
            lib = C.CDLL(_build.LIB)
            vp = C.c_void_p
            lib.fibar_default_params.argtypes = [C.POINTER(FibarParams)]
            lib.fibar_default_params.restype = None
            lib.fibar_create.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(FibarParams), C.POINTER(vp)]
            lib.fibar_create.restype = C.c_int
            lib.fibar_push_events.argtypes = [vp, vp, C.c_size_t, C.c_int, vp]
            lib.fibar_push_events.restype = C.c_int
            lib.fibar_readout.argtypes = [vp, C.c_uint64, vp, C.c_int, vp]
            lib.fibar_readout.restype = C.c_int
            lib.fibar_flush.argtypes = [vp, vp]
            lib.fibar_flush.restype = C.c_int
            lib.fibar_debug_state.argtypes = [vp, C.POINTER(FibarStateView), vp]
            lib.fibar_debug_state.restype = C.c_int
            lib.fibar_stats.argtypes = [vp, C.POINTER(FibarStats), vp]
            lib.fibar_stats.restype = C.c_int
            lib.fibar_set_timing.argtypes = [vp, C.c_int]
            lib.fibar_set_timing.restype = C.c_int
            lib.fibar_stage_times.argtypes = [vp, C.POINTER(FibarStageTimes), C.c_int, vp]
            lib.fibar_stage_times.restype = C.c_int
            lib.fibar_last_error.argtypes = [vp]
            lib.fibar_last_error.restype = C.c_char_p
            lib.fibar_destroy.argtypes = [vp]
            lib.fibar_destroy.restype = None
            lib.fibar_queue_counts_noalloc.argtypes = [vp, vp, C.c_int, vp]
            lib.fibar_queue_counts_noalloc.restype = C.c_int
            lib.fibar_readout_batch.argtypes = [C.POINTER(vp), C.POINTER(C.c_uint64), C.POINTER(vp), C.c_size_t,
                                                C.POINTER(vp), C.POINTER(C.c_int), vp]
            lib.fibar_readout_batch.restype = C.c_int
            lib.fibar_memory_bytes.argtypes = [C.c_uint32, C.c_uint32, C.POINTER(FibarParams), C.POINTER(C.c_uint64)]
            lib.fibar_memory_bytes.restype = C.c_int
            lib.fibar_relative_thresholds.argtypes = [vp, C.c_size_t, C.c_uint32, C.c_uint32, C.c_int, vp, vp, vp, vp]
            lib.fibar_relative_thresholds.restype = C.c_int
            lib.fibar_set_pixel_gain.argtypes = [vp, vp, C.c_int, vp]
            lib.fibar_set_pixel_gain.restype = C.c_int
            lib.fibar_debug_wait_timeout.argtypes = [vp, C.c_uint32, vp]
            lib.fibar_debug_wait_timeout.restype = C.c_int
            lib.fibar_push_events_many.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_size_t), C.c_size_t, C.c_int, vp]
            lib.fibar_push_events_many.restype = C.c_int
            lib.fibar_set_grid_share.argtypes = [vp, C.c_uint32]
            lib.fibar_set_grid_share.restype = C.c_int
            lib.fibar_push_batch.argtypes = [vp, vp, vp, C.c_size_t, C.c_int, vp, vp]
            lib.fibar_push_batch.restype = C.c_int
            lib.fibar_group_create.argtypes = [C.POINTER(vp), C.c_size_t, C.POINTER(vp)]
            lib.fibar_group_create.restype = C.c_int
            lib.fibar_group_readout.argtypes = [vp, vp, vp, vp, C.c_size_t, vp, vp, vp]
            lib.fibar_group_readout.restype = C.c_int
            lib.fibar_group_join.argtypes = [vp, vp]
            lib.fibar_group_join.restype = C.c_int
            lib.fibar_group_latency.argtypes = [vp, C.c_uint64, vp, C.c_size_t]
            lib.fibar_group_latency.restype = C.c_int
            lib.fibar_group_stats.argtypes = [vp, C.POINTER(FibarGroupStats)]
            lib.fibar_group_stats.restype = C.c_int
            lib.fibar_group_last_error.argtypes = [vp]
            lib.fibar_group_last_error.restype = C.c_char_p
            lib.fibar_group_destroy.argtypes = [vp]
            lib.fibar_group_destroy.restype = None
            lib.fibar_readout_host_async.argtypes = [vp, C.c_uint64, vp, vp]
            lib.fibar_readout_host_async.restype = C.c_int
            lib.fibar_wait.argtypes = [vp, vp]
            lib.fibar_wait.restype = C.c_int
            lib.fibar_fill_set_weights.argtypes = [vp, vp, C.c_size_t]
            lib.fibar_fill_set_weights.restype = C.c_int
            lib.fibar_fill_features.argtypes = [vp, vp, vp, vp]
            lib.fibar_fill_features.restype = C.c_int
            lib.fibar_fill_forward.argtypes = [vp, vp, vp, C.c_uint32, C.c_uint32, vp, vp]
            lib.fibar_fill_forward.restype = C.c_int
            lib.fibar_fill_train_step.argtypes = [vp, vp, vp, C.c_uint32, C.c_uint32, C.c_uint32, vp, C.c_uint32,
                                                  vp, vp, vp, vp, C.c_uint32, C.c_float, vp, vp]
            lib.fibar_fill_train_step.restype = C.c_int
            _lib = lib
    return _lib


# --- C-named entry points ------------------------------------------------------------

def fibar_default_params() -> FibarParams:
    p = FibarParams()
    load_library().fibar_default_params(C.byref(p))
    return p


def fibar_create(W: int, H: int, params: FibarParams | None):
    h = C.c_void_p()
    rc = load_library().fibar_create(W, H, C.byref(params) if params is not None else None, C.byref(h))
    return rc, h


def fibar_push_events(h, ev_ptr: int, n: int, on_device: int, stream: int) -> int:
    return load_library().fibar_push_events(h, ev_ptr, n, on_device, stream)


def fibar_readout(h, t_us: int, out_ptr: int, on_device: int, stream: int) -> int:
    return load_library().fibar_readout(h, t_us, out_ptr, on_device, stream)


def fibar_flush(h, stream: int) -> int:
    return load_library().fibar_flush(h, stream)


def fibar_debug_state(h, view: FibarStateView, stream: int) -> int:
    return load_library().fibar_debug_state(h, C.byref(view), stream)


def fibar_stats(h, st: FibarStats, stream: int) -> int:
    return load_library().fibar_stats(h, C.byref(st), stream)


def fibar_set_timing(h, enable: int) -> int:
    return load_library().fibar_set_timing(h, enable)


def fibar_stage_times(h, t: FibarStageTimes, reset: int, stream: int) -> int:
    return load_library().fibar_stage_times(h, C.byref(t), reset, stream)


def fibar_last_error(h) -> str:
    return load_library().fibar_last_error(h).decode()


def fibar_destroy(h) -> None:
    load_library().fibar_destroy(h)


def fibar_queue_counts_noalloc(h, cnt_ptr: int, on_device: int, stream: int) -> int:
    return load_library().fibar_queue_counts_noalloc(h, cnt_ptr, on_device, stream)


def fibar_readout_batch(hs, t_us, outs, done_events, status, stream: int) -> int:
    """hs, outs, done_events: sequences of raw pointers (ints or None); t_us: ints;
    status: a ctypes c_int array of len(hs), or None."""
    n = len(hs)
    H = (C.c_void_p * n)(*hs)
    T = (C.c_uint64 * n)(*t_us)
    O = (C.c_void_p * n)(*outs)
    D = (C.c_void_p * n)(*done_events) if done_events is not None else None
    return load_library().fibar_readout_batch(H, T, O, n, D, status, stream)


def fibar_memory_bytes(W: int, H: int, params: FibarParams | None):
    b = C.c_uint64()
    rc = load_library().fibar_memory_bytes(W, H, C.byref(params) if params is not None else None, C.byref(b))
    return rc, int(b.value)


def fibar_relative_thresholds(ev_ptr: int, n: int, W: int, H: int, on_device: int, c_on_ptr: int,
                              c_off_ptr: int, c_ptr: int, stream: int) -> int:
    return load_library().fibar_relative_thresholds(ev_ptr, n, W, H, on_device, c_on_ptr, c_off_ptr, c_ptr, stream)


def fibar_set_pixel_gain(h, gain_ptr, on_device: int, stream: int) -> int:
    return load_library().fibar_set_pixel_gain(h, gain_ptr, on_device, stream)


def fibar_push_events_many(h, ev_ptrs, ns, on_device: int, stream: int) -> int:
    n = len(ev_ptrs)
    return load_library().fibar_push_events_many(h, (C.c_void_p * n)(*ev_ptrs), (C.c_size_t * n)(*ns), n,
                                                 on_device, stream)


def fibar_debug_wait_timeout(h, max_spins: int, stream: int) -> int:
    return load_library().fibar_debug_wait_timeout(h, max_spins, stream)


def fibar_set_grid_share(h, sms: int) -> int:
    return load_library().fibar_set_grid_share(h, sms)


def fibar_push_batch(hs_ptr: int, evs_ptr: int, ns_ptr: int, count: int, on_device: int, status_ptr,
                     stream: int) -> int:
    """Arrays by address: count handles, event-packet pointers (uint64) and sizes (size_t)."""
    return load_library().fibar_push_batch(hs_ptr, evs_ptr, ns_ptr, count, on_device, status_ptr, stream)


def fibar_group_create(hs):
    g = C.c_void_p()
    n = len(hs)
    rc = load_library().fibar_group_create((C.c_void_p * n)(*hs), n, C.byref(g))
    return rc, g


def fibar_group_readout(g, members_ptr: int, t_ptr: int, outs_ptr: int, m: int, status_ptr, ticket_ptr,
                        stream: int) -> int:
    """Arrays by address: m uint32 member indices, uint64 times and image pointers."""
    return load_library().fibar_group_readout(g, members_ptr, t_ptr, outs_ptr, m, status_ptr, ticket_ptr, stream)


def fibar_group_join(g, stream: int) -> int:
    return load_library().fibar_group_join(g, stream)


def fibar_group_latency(g, ticket: int, ms_ptr: int, m: int) -> int:
    return load_library().fibar_group_latency(g, ticket, ms_ptr, m)


def fibar_group_stats(g, st: FibarGroupStats) -> int:
    return load_library().fibar_group_stats(g, C.byref(st))


def fibar_group_last_error(g) -> str:
    return load_library().fibar_group_last_error(g).decode()


def fibar_group_destroy(g) -> None:
    load_library().fibar_group_destroy(g)


def fibar_readout_host_async(h, t_us: int, out_ptr: int, stream: int) -> int:
    return load_library().fibar_readout_host_async(h, t_us, out_ptr, stream)


def fibar_wait(h, stream: int) -> int:
    return load_library().fibar_wait(h, stream)


def fibar_fill_set_weights(h, theta_ptr, n: int) -> int:
    return load_library().fibar_fill_set_weights(h, theta_ptr, n)


def fibar_fill_features(h, x_ptr: int, stale_ptr, stream: int) -> int:
    return load_library().fibar_fill_features(h, x_ptr, stale_ptr, stream)


def fibar_fill_forward(theta_ptr: int, x_ptr: int, stale_ptr: int, W: int, H: int, out_ptr: int, stream: int) -> int:
    return load_library().fibar_fill_forward(theta_ptr, x_ptr, stale_ptr, W, H, out_ptr, stream)


def fibar_fill_train_step(X, T, M, W, H, F, crops, n_crops, theta, m, v, grad, step, lr, loss_acc, stream) -> int:
    return load_library().fibar_fill_train_step(X, T, M, W, H, F, crops, n_crops, theta, m, v, grad, step, lr,
                                                loss_acc, stream)


# --- convenience wrapper ---------------------------------------------------------------

class Fibar:
    """One event stream.  Events are (n, 2) int64 tensors in the 16-byte record layout
    (``eventsim.pack_events``); CUDA tensors are pushed in place, CPU tensors copied."""

    def __init__(self, W: int, H: int, stream=None, **params):
        import torch
        if not torch.cuda.is_available():
            raise FibarError(FIBAR_ECUDA, "no CUDA device: the FIBAR library has no CPU path")
        self.torch = torch
        self.W, self.H = int(W), int(H)
        p = fibar_default_params()
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k!r}")
            setattr(p, k, v)
        self.params = p
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        rc, h = fibar_create(self.W, self.H, p)
        if rc != 0:
            raise FibarError(rc, "fibar_create failed")
        self.h = h
        self._keep = []       # device packets referenced by the pending read-out
        self._keep_prev = []  # packets of the previous read-out (may still be in flight)

    def _check(self, rc: int):
        if rc != 0:
            raise FibarError(rc, fibar_last_error(self.h))

    @property
    def _s(self) -> int:
        return self.stream.cuda_stream

    def close(self):
        if getattr(self, "h", None):
            fibar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, ev) -> None:
        t = self.torch
        if ev.dtype != t.int64 or ev.dim() != 2 or ev.shape[1] != 2 or not ev.is_contiguous():
            raise TypeError("events must be a contiguous (n, 2) int64 tensor")
        n = ev.shape[0]
        if ev.is_cuda:
            self._check(fibar_push_events(self.h, ev.data_ptr(), n, 1, self._s))
            self._keep.append(ev)
        else:
            self._check(fibar_push_events(self.h, ev.data_ptr(), n, 0, self._s))
            if ev.is_pinned():  # copied asynchronously: keep it until its read-out has run
                self._keep.append(ev)

    def push_many(self, packets) -> None:
        """Push several packets in one call (``fibar_push_events_many``): all CUDA or all CPU
        contiguous (n, 2) int64 tensors; packets adjacent in memory go in as one."""
        t = self.torch
        if not packets:
            return
        cuda = packets[0].is_cuda
        for ev in packets:
            if (ev.dtype != t.int64 or ev.dim() != 2 or ev.shape[1] != 2 or not ev.is_contiguous()
                    or ev.is_cuda != cuda):
                raise TypeError("packets must be contiguous (n, 2) int64 tensors on one device type")
        self._check(fibar_push_events_many(self.h, [ev.data_ptr() for ev in packets],
                                           [ev.shape[0] for ev in packets], 1 if cuda else 0, self._s))
        if cuda or packets[0].is_pinned():
            self._keep.extend(packets)

    def _rotate(self):
        self._keep_prev = self._keep
        self._keep = []

    def readout(self, t_us: int, out=None):
        """Image at time t_us.  ``out``: a (H, W) float32 tensor (CUDA: asynchronous,
        CPU: synchronous); default a new CUDA tensor."""
        t = self.torch
        if out is None:
            out = t.empty((self.H, self.W), dtype=t.float32, device="cuda")
        if out.dtype != t.float32 or out.numel() != self.W * self.H or not out.is_contiguous():
            raise TypeError("out must be a contiguous float32 tensor with W*H elements")
        rc = fibar_readout(self.h, int(t_us), out.data_ptr(), 1 if out.is_cuda else 0, self._s)
        self._rotate()
        self._check(rc)
        return out

    def readout_host_async(self, t_us: int, out) -> None:
        """Queue the read-out at t_us and the copy of its image into ``out`` (a contiguous
        float32 CPU tensor of W*H elements, pinned for an asynchronous copy); the image is
        there once the stream has passed it (``wait``)."""
        t = self.torch
        if out.dtype != t.float32 or out.numel() != self.W * self.H or not out.is_contiguous() or out.is_cuda:
            raise TypeError("out must be a contiguous float32 CPU tensor with W*H elements")
        rc = fibar_readout_host_async(self.h, int(t_us), out.data_ptr(), self._s)
        self._rotate()
        self._check(rc)

    def set_grid_share(self, sms: int) -> None:
        """Size the handle's kernel grids for `sms` SMs (0: the whole device)."""
        self._check(fibar_set_grid_share(self.h, int(sms)))

    def wait(self) -> None:
        self._check(fibar_wait(self.h, self._s))

    def flush(self) -> None:
        rc = fibar_flush(self.h, self._s)
        self._rotate()
        self._check(rc)

    def set_timing(self, enable: bool) -> None:
        self._check(fibar_set_timing(self.h, 1 if enable else 0))

    def stage_times(self, reset: bool = False) -> dict:
        t = FibarStageTimes()
        self._check(fibar_stage_times(self.h, t, 1 if reset else 0, self._s))
        d = {name: float(t.ms[i]) for i, name in enumerate(STAGES)}
        d["calls"] = int(t.calls)
        return d

    def stats(self) -> dict:
        st = FibarStats()
        self._check(fibar_stats(self.h, st, self._s))
        return {n: int(getattr(st, n)) for n, _ in FibarStats._fields_}

    def queue_counts_noalloc(self, out=None):
        """Queued events per pixel into ``out`` (a contiguous int32/uint32-sized tensor of
        W*H elements, CUDA or CPU; default a new CUDA int32 tensor), allocating nothing
        inside the library."""
        t = self.torch
        if out is None:
            out = t.empty((self.H, self.W), dtype=t.int32, device="cuda")
        if out.dtype != t.int32 or out.numel() != self.W * self.H or not out.is_contiguous():
            raise TypeError("out must be a contiguous int32 tensor with W*H elements")
        self._check(fibar_queue_counts_noalloc(self.h, out.data_ptr(), 1 if out.is_cuda else 0, self._s))
        return out

    def set_pixel_gain(self, gain) -> None:
        """Sec. 5.2 correction: multiply Eq. 6's right-hand side of every pixel by its gain
        (a W*H float32 tensor, CUDA or CPU); None removes it."""
        t = self.torch
        if gain is None:
            self._check(fibar_set_pixel_gain(self.h, None, 0, self._s))
            return
        if gain.dtype != t.float32 or gain.numel() != self.W * self.H or not gain.is_contiguous():
            raise TypeError("gain must be a contiguous float32 tensor with W*H elements")
        self._check(fibar_set_pixel_gain(self.h, gain.data_ptr(), 1 if gain.is_cuda else 0, self._s))
        if gain.is_cuda:
            self._keep.append(gain)

    def set_fill_weights(self, theta) -> None:
        """Learned-fill network of a blur_mode = 2 handle (FIBAR_FILL_NPARAMS floats, host
        array or CPU tensor); None returns to the Gaussian."""
        if theta is None:
            self._check(fibar_fill_set_weights(self.h, None, 0))
            return
        a = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).reshape(-1))
        self._check(fibar_fill_set_weights(self.h, a.ctypes.data, a.size))

    def fill_features(self):
        """(x [2, H, W] float32, stale [H, W] uint8) CUDA tensors of the current state."""
        t = self.torch
        x = t.empty((2, self.H, self.W), dtype=t.float32, device="cuda")
        st = t.empty((self.H, self.W), dtype=t.uint8, device="cuda")
        self._check(fibar_fill_features(self.h, x.data_ptr(), st.data_ptr(), self._s))
        return x, st

    def memory_bytes(self) -> int:
        """Device bytes this handle allocated (fibar_memory_bytes of its parameters)."""
        rc, b = fibar_memory_bytes(self.W, self.H, self.params)
        self._check(rc)
        return b

    def state(self) -> dict:
        npix = self.W * self.H
        ntiles = ((self.W + 1) // 2) * ((self.H + 1) // 2)
        arrs = dict(pbar=np.empty(npix, np.float32), L=np.empty(npix, np.float32),
                    cnt=np.empty(npix, np.uint32), tcnt=np.empty(ntiles, np.uint8),
                    stale=np.empty(npix, np.uint8), last_idx=np.empty(npix, np.uint64))
        v = FibarStateView(**{k: a.ctypes.data for k, a in arrs.items()})
        self._check(fibar_debug_state(self.h, v, self._s))
        out = dict(arrs)
        for k in ["k", "h", "q", "q_targ", "n_ap", "n_at"]:
            out[k] = int(getattr(v, k))
        return out


def memory_bytes(W: int, H: int, **params) -> int:
    """Device bytes a handle for a W x H sensor with these parameters allocates (host
    arithmetic in the library; needs no device)."""
    p = fibar_default_params()
    for k, v in params.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    rc, b = fibar_memory_bytes(int(W), int(H), p)
    if rc != 0:
        raise FibarError(rc, "fibar_memory_bytes rejected the arguments")
    return b


def readout_batch(fibars, t_us, outs=None, done_events=None, stream=None):
    """Read out several :class:`Fibar` handles together (``fibar_readout_batch``).

    ``outs``: CUDA float32 tensors of each handle's W*H (default: new ones);
    ``done_events``: optional ``torch.cuda.Event`` per handle (or None entries), each
    recorded when that handle's image is complete.  Returns the list of images; raises
    :class:`FibarError` naming the first failing handle."""
    import torch
    n = len(fibars)
    if len(t_us) != n:
        raise ValueError("one read-out time per handle")
    if outs is None:
        outs = [torch.empty((f.H, f.W), dtype=torch.float32, device="cuda") for f in fibars]
    for f, o in zip(fibars, outs):
        if (o.dtype != torch.float32 or not o.is_cuda or o.numel() != f.W * f.H
                or not o.is_contiguous()):
            raise TypeError("outs must be contiguous CUDA float32 tensors of W*H elements")
    ev_ptrs = None
    if done_events is not None:
        ev_ptrs = []
        for ev in done_events:
            if ev is None:
                ev_ptrs.append(None)
                continue
            if not ev.cuda_event:  # created lazily by torch: make it exist
                ev.record()
            ev_ptrs.append(ev.cuda_event)
    s = stream if stream is not None else torch.cuda.current_stream()
    status = (C.c_int * n)()
    rc = fibar_readout_batch([f.h.value for f in fibars], [int(t) for t in t_us],
                             [o.data_ptr() for o in outs], ev_ptrs, status, s.cuda_stream)
    for f in fibars:
        f._rotate()
    if rc != 0:
        for i, f in enumerate(fibars):
            if status[i] != 0:
                raise FibarError(status[i], f"handle {i}: {fibar_last_error(f.h)}")
        raise FibarError(rc, "fibar_readout_batch rejected the arguments")
    return outs


def push_batch(fibars, packets, stream=None) -> None:
    """Push device packets to several handles in one call (``fibar_push_batch``):
    ``packets[k]`` (a contiguous CUDA (n, 2) int64 tensor) goes to ``fibars[k]``; a handle
    may appear more than once (its packets in order)."""
    import torch
    n = len(fibars)
    if len(packets) != n:
        raise ValueError("one packet per entry")
    hs = np.empty(n, np.uint64)
    ptrs = np.empty(n, np.uint64)
    ns = np.empty(n, np.uint64)
    for k, (f, ev) in enumerate(zip(fibars, packets)):
        if not ev.is_cuda or ev.dtype != torch.int64 or ev.dim() != 2 or ev.shape[1] != 2 or not ev.is_contiguous():
            raise TypeError("packets must be contiguous CUDA (n, 2) int64 tensors")
        hs[k] = f.h.value
        ptrs[k] = ev.data_ptr()
        ns[k] = ev.shape[0]
    _push_arrays(fibars, packets, hs, ptrs, ns, stream)


def _push_arrays(fibars, keep, hs, ptrs, ns, stream=None):
    _push_lists(fibars, keep, hs.tolist(), ptrs.tolist(), ns.tolist(), stream)


def _push_lists(fibars, keep, hs, ptrs, ns, stream=None):
    """fibar_push_batch of device packets given as lists of handle integers, packet
    addresses and sizes; keeps each packet's tensor (``keep``) with its handle."""
    import torch
    n = len(hs)
    a_h, a_p, a_n = array.array("Q", hs), array.array("Q", ptrs), array.array("Q", ns)
    status = array.array("i", bytes(4 * n))
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = fibar_push_batch(a_h.buffer_info()[0], a_p.buffer_info()[0], a_n.buffer_info()[0], n, 1,
                          status.buffer_info()[0], s.cuda_stream)
    for f, ev in zip(fibars, keep):
        k = f._keep
        if not k or k[-1] is not ev:
            k.append(ev)
    if rc != 0:
        k = next((i for i in range(n) if status[i] != 0), 0)
        raise FibarError(rc, f"entry {k}: {fibar_last_error(fibars[k].h)}")


class Group:
    """A fixed set of :class:`Fibar` handles, each member's read-out one launch of its
    captured graph on the member's own stream (``fibar_group_*``).  Images are complete
    once ``join`` has ordered a stream after them (or ``latency_ms`` has waited).  Destroy
    (``close``) before the handles."""

    def __init__(self, fibars):
        if not fibars:
            raise ValueError("a group needs at least one handle")
        self.fibars = list(fibars)
        rc, g = fibar_group_create([f.h.value for f in self.fibars])
        if rc != 0:
            raise FibarError(rc, "fibar_group_create failed")
        self.g = g
        self._tickets = {}

    def _check(self, rc: int):
        if rc != 0:
            raise FibarError(rc, fibar_group_last_error(self.g))

    def readout(self, members, t_us, outs, stream=None) -> int:
        """Read out members (indices into the group) at t_us into outs (16-byte aligned
        contiguous CUDA float32 tensors of each member's W*H); returns the call's ticket."""
        import torch
        m = len(members)
        if len(t_us) != m or len(outs) != m:
            raise ValueError("one time and one output per member")
        for i, o in zip(members, outs):
            f = self.fibars[i]
            if o.dtype != torch.float32 or not o.is_cuda or o.numel() != f.W * f.H or not o.is_contiguous():
                raise TypeError("outs must be contiguous CUDA float32 tensors of W*H elements")
        s = stream if stream is not None else torch.cuda.current_stream()
        return self.readout_ptrs(members, t_us, [o.data_ptr() for o in outs], s.cuda_stream)

    def readout_ptrs(self, members, t_us, out_ptrs, cuda_stream: int) -> int:
        """``readout`` with the images as device addresses (each W*H floats of its member)
        and the stream as a raw handle: no tensor checks, for callers that made the
        images themselves."""
        m = len(members)
        mem = array.array("I", members)
        ts = array.array("Q", t_us)
        op = array.array("Q", out_ptrs)
        status = array.array("i", bytes(4 * m))
        ticket = array.array("Q", [0])
        rc = fibar_group_readout(self.g, mem.buffer_info()[0], ts.buffer_info()[0], op.buffer_info()[0], m,
                                 status.buffer_info()[0], ticket.buffer_info()[0], cuda_stream)
        if rc != 0:
            bad = [k for k in range(m) if status[k] != 0]
            if bad:
                i = int(members[bad[0]])
                detail = fibar_last_error(self.fibars[i].h) if 0 <= i < len(self.fibars) else ""
                raise FibarError(rc, f"entry {bad[0]}: {fibar_group_last_error(self.g)} {detail}")
            self._check(rc)
        fibars = self.fibars
        for i in members:
            fibars[i]._rotate()
        return ticket[0]

    def join(self, stream=None) -> None:
        """Make later work on ``stream`` (default: the current stream) wait for every read-out
        queued so far."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        self._check(fibar_group_join(self.g, s.cuda_stream))

    def latency_ms(self, ticket: int, m: int):
        """Device ms from the launch's start to each of its m images (waits)."""
        ms = np.zeros(m, np.float32)
        self._check(fibar_group_latency(self.g, int(ticket), ms.ctypes.data, m))
        return [float(x) for x in ms]

    def stats(self) -> dict:
        st = FibarGroupStats()
        self._check(fibar_group_stats(self.g, st))
        return {k: int(getattr(st, k)) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "g", None):
            fibar_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def relative_thresholds(ev, W: int, H: int, stream=None):
    """(c_on, c_off, c) relative thresholds of a calibration recording, as (H, W) float32
    tensors on the events' device (``fibar_relative_thresholds``)."""
    import torch
    if ev.dtype != torch.int64 or ev.dim() != 2 or ev.shape[1] != 2 or not ev.is_contiguous():
        raise TypeError("events must be a contiguous (n, 2) int64 tensor")
    outs = [torch.empty((H, W), dtype=torch.float32, device=ev.device) for _ in range(3)]
    s = 0
    if ev.is_cuda:
        s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    rc = fibar_relative_thresholds(ev.data_ptr(), ev.shape[0], int(W), int(H), 1 if ev.is_cuda else 0,
                                   *[o.data_ptr() for o in outs], s)
    if rc != 0:
        raise FibarError(rc, "fibar_relative_thresholds failed")
    return tuple(outs)


def fill_forward(theta, x, stale, stream=None):
    """The learned fill of explicit inputs (x [2, H, W] float32 and stale [H, W] uint8 CUDA
    tensors) with the read-out's kernel: a new [H, W] CUDA float32 image."""
    import torch
    if not (x.is_cuda and stale.is_cuda and x.dtype == torch.float32 and stale.dtype == torch.uint8
            and x.dim() == 3 and x.shape[0] == 2 and tuple(stale.shape) == tuple(x.shape[1:])
            and x.is_contiguous() and stale.is_contiguous()):
        raise TypeError("x must be a contiguous CUDA float32 [2, H, W] tensor and stale a uint8 [H, W] one")
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).reshape(-1))
    if th.size != FIBAR_FILL_NPARAMS:
        raise ValueError(f"theta must have {FIBAR_FILL_NPARAMS} parameters")
    H, W = int(x.shape[1]), int(x.shape[2])
    out = torch.empty((H, W), dtype=torch.float32, device=x.device)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    rc = fibar_fill_forward(th.ctypes.data, x.data_ptr(), stale.data_ptr(), W, H, out.data_ptr(), s)
    if rc != 0:
        raise FibarError(rc, "fibar_fill_forward failed")
    return out

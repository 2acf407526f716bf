"""Serving many FIBAR streams from one process: device-resident state, admission by
device memory, and read-out requests answered in concurrent batches.

The paper reconstructs one camera and states that an image can be read out at any time
(Sec. 1).  A server holds one library handle per admitted stream (its filter state, queue
and rings stay in device memory between calls), pushes each stream's packets as they
arrive, and answers read-out requests for arbitrary times.  The requests that are due are
served together: by default as one launch of a group graph (``fibar_group_readout``: every
admitted stream's read-out chain captured once, the streams read out chosen per launch),
else through ``fibar_readout_batch`` (each chain launched from the host onto a pool of
streams).  Either way the pipelines of different streams run side by side on the GPU.  A
request's latency is the device time from its batch's start to its image being complete
(group: the kernels' own timer stamps; batch: CUDA events).

:class:`Admission` is the memory accounting alone (host logic, no device), so that its
rules can be checked without a GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .binding import Fibar, FibarError, Group, _push_lists, memory_bytes, readout_batch

# per handle, on top of the library's count: the driver's allocation granularity
HANDLE_SLACK_BYTES = 8 << 20


class Admission:
    """Admit streams while their device memory fits a budget.

    ``budget``: bytes the server may hold.  ``bytes_fn(W, H, **params)``: the bytes a
    handle needs (default: the library's ``fibar_memory_bytes``) plus a fixed slack."""

    def __init__(self, budget: int, bytes_fn=None, slack: int = HANDLE_SLACK_BYTES):
        if budget < 0:
            raise ValueError("budget must be >= 0")
        self.budget = int(budget)
        self.bytes_fn = bytes_fn or memory_bytes
        self.slack = int(slack)
        self.held: dict[int, int] = {}
        self.refused = 0
        self._next = 0

    @property
    def used(self) -> int:
        return sum(self.held.values())

    def need(self, W: int, H: int, **params) -> int:
        return int(self.bytes_fn(W, H, **params)) + self.slack

    def try_admit(self, W: int, H: int, **params):
        """The new stream's id, or None (refused) if it does not fit."""
        need = self.need(W, H, **params)
        if self.used + need > self.budget:
            self.refused += 1
            return None
        sid = self._next
        self._next += 1
        self.held[sid] = need
        return sid

    def release(self, sid: int) -> None:
        self.held.pop(sid)


@dataclass
class Request:
    sid: int
    t_us: int
    image: object = None      # CUDA (H, W) float32 tensor, valid once its batch has run
    done: object = None       # batch path: torch.cuda.Event recorded when the image is complete
    start: object = None      # batch path: torch.cuda.Event recorded before the batch
    group: object = None      # group path: the Group whose launch served it
    ticket: int = -1          # group path: that launch's ticket
    k: int = -1               # group path: this request's entry in that launch
    m: int = 0                # group path: entries in that launch


@dataclass
class _Stream:
    fib: Fibar
    W: int
    H: int
    last_t: int = -1
    queue: list = field(default_factory=list)  # pending Requests, in arrival order
    hval: int = 0                               # the library handle, as an integer


class GridTuner:
    """Chooses, per sensor shape, how many SMs a stream's kernels are sized for
    (``fibar_set_grid_share``) when many streams are read out concurrently.

    For a shape, ``tune`` reads out ``n_streams`` handles of that shape together
    (``fibar_readout_batch``), each applying ``events_per_readout`` simulated events per
    read-out, with every candidate share in turn, times the rounds with CUDA events and
    keeps the share with the most events per second.  The choices are recorded in
    ``table`` ((W, H) -> SMs, 0 = the whole device) and ``trials`` (the timings)."""

    def __init__(self, candidates=None, rounds: int = 3, warm: int = 1, seed: int = 31, use_graph: bool = True):
        import torch
        self.torch = torch
        self.use_graph = use_graph
        self.sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        # the whole device, then a quarter down to a twelfth (on the 32-stream workload a
        # quarter or an eighth won on every sensor; half of the device never did)
        self.candidates = candidates or [0, self.sms // 4, self.sms // 6, self.sms // 8, self.sms // 12]
        self.rounds, self.warm, self.seed = rounds, warm, seed
        self.table: dict[tuple[int, int], int] = {}
        self.trials: dict[tuple[int, int], list] = {}

    def tune(self, W: int, H: int, n_streams: int, events_per_readout: int, **params) -> int:
        import eventsim
        torch = self.torch
        per = max(1024, int(events_per_readout))
        total = per * (self.warm + self.rounds) * len(self.candidates)
        fibs = [Fibar(W, H, **params) for _ in range(n_streams)]
        evs = [eventsim.simulate(W, H, total, scene="perlin", seed=self.seed + i, noise_frac=0.02, device="cuda")
               for i in range(n_streams)]
        stream = torch.cuda.current_stream()
        trials = []
        pos = 0
        group = Group(fibs) if self.use_graph else None
        outs = [torch.empty((H, W), dtype=torch.float32, device="cuda") for _ in fibs]
        tcols = [ev[:, 1].cpu() for ev in evs]
        members = list(range(n_streams))
        try:
            for sms in self.candidates:
                for f in fibs:
                    f.set_grid_share(sms)
                t0 = t1 = None
                for r in range(self.warm + self.rounds):
                    if r == self.warm:
                        t0 = torch.cuda.Event(enable_timing=True)
                        t0.record(stream)
                    for f, ev in zip(fibs, evs):
                        f.push(ev[pos:pos + per])
                    ts = [int(tc[pos + per - 1]) for tc in tcols]
                    if group is not None:
                        group.readout(members, ts, outs, stream=stream)
                    else:
                        readout_batch(fibs, ts, outs, stream=stream)
                    pos += per
                if group is not None:
                    group.join(stream)
                t1 = torch.cuda.Event(enable_timing=True)
                t1.record(stream)
                t1.synchronize()
                ms = t0.elapsed_time(t1)
                trials.append({"sms": sms, "ms": round(ms, 4),
                               "mev_s": round(n_streams * per * self.rounds / ms / 1e3, 2)})
        finally:
            if group is not None:
                group.close()
            for f in fibs:
                f.close()
        best = max(trials, key=lambda t: t["mev_s"])["sms"]
        self.table[(W, H)] = best
        self.trials[(W, H)] = trials
        return best


class Server:
    """Device-resident FIBAR streams behind one loop.

    ``budget``: device bytes for stream state (default: the free memory reported by
    ``torch.cuda.mem_get_info`` minus ``reserve``)."""

    def __init__(self, budget: int | None = None, reserve: int = 4 << 30, stream=None, use_graph: bool = True):
        import torch
        self.torch = torch
        self.use_graph = use_graph
        self.group = None        # Group over the admitted streams (rebuilt after admit/release)
        self._members = {}       # sid -> index in the group
        self._old_groups = []    # replaced groups, kept for their tickets until close()
        self._ev_cache = {}      # id(events tensor) -> (tensor, data_ptr, rows), for push_ranges
        if budget is None:
            free, _ = torch.cuda.mem_get_info()
            budget = max(0, free - reserve)
        self.admission = Admission(budget)
        self.streams: dict[int, _Stream] = {}
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.batches = 0
        self.grid_share: dict[tuple[int, int], int] = {}

    def admit(self, W: int, H: int, **params):
        """Create a stream's handle if its memory fits; returns its id or None."""
        sid = self.admission.try_admit(W, H, **params)
        if sid is None:
            return None
        try:
            fib = Fibar(W, H, stream=self.stream, **params)
        except FibarError:
            self.admission.release(sid)
            self.admission.refused += 1
            return None
        self.streams[sid] = _Stream(fib, W, H, hval=fib.h.value)
        self._drop_group()
        if (W, H) in self.grid_share:
            fib.set_grid_share(self.grid_share[(W, H)])
        return sid

    def set_grid_share(self, table: dict) -> None:
        """Per sensor shape (W, H), the SMs its streams' kernels are sized for (see
        :class:`GridTuner`); applies to admitted and future streams."""
        self.grid_share.update(table)
        for st in self.streams.values():
            if (st.W, st.H) in table:
                st.fib.set_grid_share(table[(st.W, st.H)])

    def release(self, sid: int) -> None:
        self._drop_group(close_all=True)
        st = self.streams.pop(sid)
        st.fib.close()
        self.admission.release(sid)

    def _drop_group(self, close_all: bool = False) -> None:
        self.join()
        if self.group is not None:
            self._old_groups.append(self.group)
            self.group = None
        if close_all:  # a member is about to go: its groups must go first
            for g in self._old_groups:
                g.close()
            self._old_groups = []

    def _ensure_group(self) -> Group:
        if self.group is None:
            sids = list(self.streams)
            self.group = Group([self.streams[i].fib for i in sids])
            self._members = {sid: k for k, sid in enumerate(sids)}
        return self.group

    def push(self, sid: int, packet) -> None:
        """Queue a packet (CUDA (n, 2) int64 event records) for the stream."""
        self.streams[sid].fib.push(packet)

    def push_ranges(self, items) -> None:
        """Queue several device packets in one library call: items of (sid, events, lo,
        hi), the rows lo:hi of a contiguous CUDA (n, 2) int64 tensor ``events`` (which must
        stay alive until the stream's read-out has run; the handle keeps a reference)."""
        n = len(items)
        if n == 0:
            return
        cache = self._ev_cache
        streams = self.streams
        hs, ptrs, ns, fibs, keep = [], [], [], [], []
        for sid, ev, lo, hi in items:
            st = streams[sid]
            c = cache.get(id(ev))
            if c is None or c[0] is not ev:
                if (not ev.is_cuda or ev.dtype != self.torch.int64 or ev.dim() != 2 or ev.shape[1] != 2
                        or not ev.is_contiguous()):
                    raise TypeError("events must be a contiguous CUDA (n, 2) int64 tensor")
                if len(cache) >= 256:  # bounded: it holds its tensors alive
                    cache.clear()
                c = cache[id(ev)] = (ev, ev.data_ptr(), ev.shape[0])
            if not 0 <= lo <= hi <= c[2]:
                raise ValueError("packet range outside the events")
            hs.append(st.hval)
            ptrs.append(c[1] + 16 * lo)
            ns.append(hi - lo)
            fibs.append(st.fib)
            keep.append(ev)
        _push_lists(fibs, keep, hs, ptrs, ns, self.stream)

    def request(self, sid: int, t_us: int) -> Request:
        """Ask for the stream's image at t_us (not earlier than its previous request)."""
        st = self.streams[sid]
        if t_us < st.last_t:
            raise ValueError(f"stream {sid}: read-out time {t_us} earlier than {st.last_t}")
        st.last_t = t_us
        r = Request(sid, int(t_us))
        st.queue.append(r)
        return r

    def pending(self) -> int:
        return sum(len(s.queue) for s in self.streams.values())

    def serve(self) -> list[Request]:
        """Answer every queued request: each batch takes the oldest request of every stream
        that has one, so a stream's requests are served in order.  Returns them.  With group
        read-outs an image is complete once `join()` (or `latencies_ms`) has waited for it;
        keep each Request (it holds its image) until then."""
        torch = self.torch
        served = []
        while True:
            batch = [(sid, st) for sid, st in self.streams.items() if st.queue]
            if not batch:
                return served
            reqs = [st.queue.pop(0) for _, st in batch]
            for r, (_, st) in zip(reqs, batch):
                r.image = torch.empty((st.H, st.W), dtype=torch.float32, device="cuda")
            if self.use_graph:
                g = self._ensure_group()
                members = self._members
                ticket = g.readout_ptrs([members[sid] for sid, _ in batch], [r.t_us for r in reqs],
                                        [r.image.data_ptr() for r in reqs], self.stream.cuda_stream)
                m = len(reqs)
                for k, r in enumerate(reqs):
                    r.group, r.ticket, r.k, r.m = g, ticket, k, m
            else:
                start = torch.cuda.Event(enable_timing=True)
                start.record(self.stream)
                for r in reqs:
                    r.done = torch.cuda.Event(enable_timing=True)
                    r.start = start
                readout_batch([st.fib for _, st in batch], [r.t_us for r in reqs],
                              [r.image for r in reqs], [r.done for r in reqs], stream=self.stream)
            self.batches += 1
            served.extend(reqs)

    def join(self) -> None:
        """Make later work on the server's stream wait for every read-out served so far
        (group read-outs run on the members' own streams)."""
        if self.group is not None:
            self.group.join(self.stream)
        for g in self._old_groups:
            g.join(self.stream)

    def stats(self) -> dict:
        self.join()
        out = {"streams": len(self.streams), "bytes_held": self.admission.used,
               "budget": self.admission.budget, "refused": self.admission.refused,
               "batches": self.batches, "kernel_launches": 0, "events_applied": 0}
        for st in self.streams.values():
            s = st.fib.stats()
            out["kernel_launches"] += s["kernel_launches"]
            out["events_applied"] += s["events_applied"]
        return out

    def close(self) -> None:
        self._drop_group(close_all=True)
        for sid in list(self.streams):
            self.release(sid)


def latencies_ms(requests) -> list[float]:
    """Device time from each request's batch start to its image (synchronises).  Call
    before the server that served them is closed."""
    out = []
    cache = {}
    for r in requests:
        if r.group is not None:
            key = (id(r.group), r.ticket)
            if key not in cache:
                cache[key] = r.group.latency_ms(r.ticket, r.m)
            out.append(cache[key][r.k])
        else:
            r.done.synchronize()
            out.append(r.start.elapsed_time(r.done))
    return out

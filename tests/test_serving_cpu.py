"""Host-side logic of batched serving (no GPU): memory accounting, the library's memory
query, the seeded mixed-stream inputs, and the marshalling of batched pushes."""
import numpy as np
import pytest

import eventsim


def test_admission_budget_and_release():
    from paper_2510_20071_gb300.serving import Admission
    sizes = {(10, 10): 100, (20, 20): 400}
    a = Admission(budget=1000, bytes_fn=lambda W, H, **p: sizes[(W, H)], slack=50)
    assert a.need(10, 10) == 150
    s0 = a.try_admit(20, 20)          # 450
    s1 = a.try_admit(20, 20)          # 900
    assert (s0, s1) == (0, 1) and a.used == 900
    assert a.try_admit(10, 10) is None and a.refused == 1   # 1050 > 1000
    a.release(s0)
    assert a.used == 450
    s2 = a.try_admit(10, 10)
    assert s2 == 2 and a.used == 600
    with pytest.raises(ValueError):
        Admission(budget=-1)


def test_memory_bytes_properties():
    from paper_2510_20071_gb300 import memory_bytes, FibarError
    b = {m: memory_bytes(640, 480, **p) for m, p in
         {"nsf": dict(spatial_filter=0), "s2": dict(blur_mode=1), "s1": dict(blur_mode=0)}.items()}
    assert 0 < b["nsf"] < b["s2"] < b["s1"]
    for v in b.values():
        assert v % 512 == 0
    # grows with the sensor and with the pending capacity
    assert memory_bytes(1280, 720, blur_mode=1) > memory_bytes(640, 480, blur_mode=1)
    small = memory_bytes(240, 180, blur_mode=1, max_pending=1 << 18)
    big = memory_bytes(240, 180, blur_mode=1, max_pending=1 << 22)
    # every pending event holds at least a staging record, two carry records and two
    # sort records (16 + 32 + 16 bytes)
    assert big - small >= 64 * ((1 << 22) - (1 << 18))
    # at least the per-pixel state: p_bar, L, last event index, output staging
    assert memory_bytes(1280, 720, spatial_filter=0, max_pending=1024) >= 1280 * 720 * (4 + 4 + 8 + 4)
    for bad in [dict(W=0, H=4), dict(W=4, H=4, fill_num=0), dict(W=4, H=4, max_pending=(1 << 27) + 1)]:
        W, H = bad.pop("W"), bad.pop("H")
        with pytest.raises(FibarError):
            memory_bytes(W, H, **bad)


def test_mixed_streams_and_requests_are_seeded():
    a = eventsim.mixed_streams(3, 0.002, sensors=[(64, 48), (96, 72)], rate_lo=1e6, rate_hi=3e6)
    b = eventsim.mixed_streams(3, 0.002, sensors=[(64, 48), (96, 72)], rate_lo=1e6, rate_hi=3e6)
    for x, y in zip(a, b):
        assert (x["W"], x["H"]) == (y["W"], y["H"])
        assert np.array_equal(x["events"].numpy(), y["events"].numpy())
        t = x["events"][:, 1].numpy()
        assert t[0] == 0 and t[-1] == 2000 and np.all(np.diff(t) >= 0)
        assert 1e6 * 0.002 * 0.99 <= x["events"].shape[0] <= 3e6 * 0.002 * 1.01
    r = eventsim.request_times(3, 0.002, rate_hz=5000)
    assert r == eventsim.request_times(3, 0.002, rate_hz=5000)
    for ts in r:
        assert ts[-1] == 2000 and ts == sorted(ts)


def test_serving_schedule_covers_every_event_once():
    s = eventsim.mixed_streams(2, 0.003, sensors=[(64, 48)], rate_lo=1e6, rate_hi=2e6)
    r = eventsim.request_times(2, 0.003, rate_hz=3000)
    sch = eventsim.serving_schedule(s, r, tick_us=700)
    seen = [np.zeros(d["events"].shape[0], dtype=int) for d in s]
    reads = [[] for _ in s]
    for T, pushes, rd in sch:
        for i, lo, hi in pushes:
            seen[i][lo:hi] += 1
            t = s[i]["events"][lo:hi, 1].numpy()
            assert np.all((t >= T) & (t < T + 700))
        for i, t in rd:
            assert T <= t < T + 700
            reads[i].append(t)
    assert all(np.all(x == 1) for x in seen)
    assert reads == r


class _FakeEvents:
    """Stands in for a contiguous CUDA (n, 2) int64 tensor (host logic only)."""

    def __init__(self, n, addr):
        import torch
        self.shape = (n, 2)
        self.is_cuda = True
        self.dtype = torch.int64
        self._addr = addr

    def dim(self):
        return 2

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return self._addr


def test_push_ranges_marshals_addresses_and_keeps_packets(monkeypatch):
    import torch
    from paper_2510_20071_gb300 import serving

    class Fib:
        def __init__(self, hval):
            self.h = type("H", (), {"value": hval})()
            self._keep = []

    calls = []

    def fake_push(fibs, keep, hs, ptrs, ns, stream):
        calls.append((list(hs), list(ptrs), list(ns)))
        for f, ev in zip(fibs, keep):
            if not f._keep or f._keep[-1] is not ev:
                f._keep.append(ev)

    monkeypatch.setattr(serving, "_push_lists", fake_push)
    srv = serving.Server.__new__(serving.Server)
    srv.torch = torch
    srv.stream = None
    srv._ev_cache = {}
    srv.streams = {7: serving._Stream(Fib(1000), 4, 4, hval=1000), 9: serving._Stream(Fib(2000), 4, 4, hval=2000)}
    a, b = _FakeEvents(100, 1 << 20), _FakeEvents(50, 1 << 24)
    srv.push_ranges([(7, a, 10, 30), (9, b, 0, 50), (7, a, 30, 31)])
    hs, ptrs, ns = calls[-1]
    assert hs == [1000, 2000, 1000]
    assert ptrs == [(1 << 20) + 16 * 10, 1 << 24, (1 << 20) + 16 * 30]   # 16-byte records
    assert ns == [20, 50, 1]
    assert srv.streams[7].fib._keep == [a] and srv.streams[9].fib._keep == [b]
    srv.push_ranges([])                      # nothing to do: no library call
    assert len(calls) == 1
    with pytest.raises(ValueError):
        srv.push_ranges([(7, a, 90, 101)])   # past the end of the events
    with pytest.raises(ValueError):
        srv.push_ranges([(7, a, 5, 4)])
    # the address cache stays bounded however many packet tensors go through
    for i in range(600):
        srv.push_ranges([(9, _FakeEvents(8, (i + 1) << 12), 0, 8)])
    assert len(srv._ev_cache) <= 256

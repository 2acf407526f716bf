"""Host-side logic of batched serving (no GPU): memory accounting, the library's memory
query, and the seeded mixed-stream inputs."""
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

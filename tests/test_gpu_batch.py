"""Batched serving on the GPU: fibar_readout_batch and the Server against the FP64 oracle,
one stream at a time, on seeded streams of mixed sensors with read-out requests at random
(Poisson) times."""
import ctypes as C

import numpy as np
import pytest
import torch

import eventsim
from tests.harness import compare

pytestmark = pytest.mark.gpu

MODES = {
    "nsf": dict(spatial_filter=0),
    "s1": dict(spatial_filter=1, blur_mode=0),
    "s2": dict(spatial_filter=1, blur_mode=1),
}
SENSORS = [(64, 48), (96, 72), (120, 90), (33, 17)]


def _streams(n, seconds, seed):
    return eventsim.mixed_streams(n, seconds, seed=seed, sensors=SENSORS, rate_lo=0.5e6, rate_hi=4e6)


@pytest.mark.parametrize("mode,sms,graph", [("s2", 0, True), ("s1", 0, True), ("nsf", 0, True), ("s2", 1, True),
                                            ("s1", 3, False), ("nsf", 19, True), ("s2", 0, False)])
def test_served_images_match_oracle_per_stream(oracle_mod, mode, sms, graph):
    """sms: the SMs every stream's grids are sized for (0: the whole device); graph: one
    group-graph launch per batch (else fibar_readout_batch)."""
    from paper_2510_20071_gb300.serving import Server, latencies_ms
    params = dict(MODES[mode], c_on=0.2, c_off=0.2)
    streams = _streams(6, 0.008, seed=21)
    reqs = eventsim.request_times(6, 0.008, rate_hz=2500, seed=22)
    sched = eventsim.serving_schedule(streams, reqs, tick_us=400)
    dev = [s["events"].cuda() for s in streams]
    srv = Server(use_graph=graph)
    if sms:
        srv.set_grid_share({(W, H): sms for W, H in SENSORS})
    sids = [srv.admit(s["W"], s["H"], **params) for s in streams]
    assert None not in sids
    steps = [[] for _ in streams]
    served = [[] for _ in streams]
    try:
        for T, pushes, reads in sched:
            if graph:  # the tick's packets in one library call
                srv.push_ranges([(sids[i], dev[i], lo, hi) for i, lo, hi in pushes])
            for i, lo, hi in pushes:
                if not graph:
                    srv.push(sids[i], dev[i][lo:hi])
                steps[i].append(("push", lo, hi))
            for i, t in reads:
                served[i].append(srv.request(sids[i], t))
                steps[i].append(("read", t))
            srv.serve()
        assert srv.pending() == 0
        torch.cuda.synchronize()
        lat = latencies_ms([r for rs in served for r in rs])
        assert all(x > 0 for x in lat)
        for i, s in enumerate(streams):
            W, H = s["W"], s["H"]
            o = oracle_mod.Oracle(W, H, **params)
            o_imgs = []
            for st in steps[i]:
                if st[0] == "push":
                    o.push(s["events"][st[1]:st[2]])
                else:
                    o_imgs.append(o.readout(st[1]))
            g_imgs = [r.image.cpu().numpy().astype(np.float64) for r in served[i]]
            g_state = srv.streams[sids[i]].fib.state()
            compare(W, H, o_imgs, [o.state()], g_imgs, [g_state], spatial=params["spatial_filter"] == 1)
        st = srv.stats()
        assert st["batches"] >= max(len(r) for r in reqs)
        assert st["events_applied"] == sum(s["events"].shape[0] for s in streams)
    finally:
        srv.close()


@pytest.mark.parametrize("mode", ["s2", "s1", "nsf"])
def test_grid_share_does_not_change_results(mode):
    """Every stage's result is independent of its grid (grid-stride loops, work taken
    from counters): a handle sized for 2 or 19 SMs gives the whole-device handle's
    images and state bit for bit."""
    from paper_2510_20071_gb300 import Fibar
    W, H = 346, 260
    ev = eventsim.simulate(W, H, 1_500_000, scene="perlin", seed=41, noise_frac=0.02)
    cuts = [200_000, 700_000, 1_500_000]
    params = dict(MODES[mode], c_on=0.2, c_off=0.2)
    runs = []
    for sms in (0, 2, 19):
        f = Fibar(W, H, **params)
        f.set_grid_share(sms)
        imgs, lo = [], 0
        try:
            for hi in cuts:
                f.push(ev[lo:hi].cuda())
                imgs.append(f.readout(int(ev[hi - 1, 1])).cpu())
                lo = hi
            runs.append((imgs, f.state()))
        finally:
            f.close()
    for imgs, state in runs[1:]:
        for a, b in zip(runs[0][0], imgs):
            assert torch.equal(a, b)
        for k in runs[0][1]:
            np.testing.assert_array_equal(np.asarray(runs[0][1][k]), np.asarray(state[k]), err_msg=k)


def test_grid_share_tuner_records_a_choice_per_shape():
    from paper_2510_20071_gb300.serving import GridTuner
    t = GridTuner(candidates=[0, 8], rounds=2, warm=1)
    for W, H in [(64, 48), (120, 90)]:
        best = t.tune(W, H, 3, 20_000, c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=1)
        assert best in (0, 8)
        assert t.table[(W, H)] == best
        assert [r["sms"] for r in t.trials[(W, H)]] == [0, 8]
        assert all(r["ms"] > 0 and r["mev_s"] > 0 for r in t.trials[(W, H)])


def _pushed_handles(streams, params):
    from paper_2510_20071_gb300 import Fibar
    hs = []
    for s in streams:
        f = Fibar(s["W"], s["H"], **params)
        f.push(s["events"].cuda())
        hs.append(f)
    return hs


def test_batch_status_isolates_a_failing_handle():
    from paper_2510_20071_gb300 import binding, FIBAR_EORDER
    params = dict(MODES["s2"], c_on=0.2, c_off=0.2)
    streams = _streams(3, 0.004, seed=31)
    a = _pushed_handles(streams, params)   # batched
    b = _pushed_handles(streams, params)   # one at a time
    try:
        t1 = [1000, 1500, 2000]
        outs = [torch.empty((s["H"], s["W"]), device="cuda") for s in streams]
        binding.readout_batch(a, t1, outs)
        ref = [f.readout(t) for f, t in zip(b, t1)]
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
        # handle 1 asks for a time before its previous read-out: only it fails
        t2 = [3000, 1200, 4000]
        status = (C.c_int * 3)()
        outs2 = [torch.empty_like(o) for o in outs]
        rc = binding.fibar_readout_batch([f.h.value for f in a], t2, [o.data_ptr() for o in outs2], None,
                                         status, torch.cuda.current_stream().cuda_stream)
        assert rc == FIBAR_EORDER and list(status) == [0, FIBAR_EORDER, 0]
        assert "earlier" in binding.fibar_last_error(a[1].h)
        ref2 = [b[0].readout(3000), None, b[2].readout(4000)]
        torch.cuda.synchronize()
        assert torch.equal(outs2[0], ref2[0]) and torch.equal(outs2[2], ref2[2])
        for fa, fb in zip(a, b):
            sa, sb = fa.state(), fb.state()
            assert sa["k"] == sb["k"] and sa["h"] == sb["h"]
            np.testing.assert_array_equal(sa["L"], sb["L"])
    finally:
        for f in a + b:
            f.close()


def test_batch_rejects_bad_arguments_before_any_work():
    from paper_2510_20071_gb300 import binding, FIBAR_EINVAL
    params = dict(MODES["s2"], c_on=0.2, c_off=0.2)
    streams = _streams(2, 0.002, seed=41)
    a = _pushed_handles(streams, params)
    try:
        outs = [torch.empty((s["H"], s["W"]), device="cuda") for s in streams]
        s = torch.cuda.current_stream().cuda_stream
        status = (C.c_int * 2)(7, 7)
        dup = [a[0].h.value, a[0].h.value]
        rc = binding.fibar_readout_batch(dup, [10, 20], [o.data_ptr() for o in outs], None, status, s)
        assert rc == FIBAR_EINVAL and list(status) == [7, 7]
        assert all(f.state()["k"] == 0 for f in a)
        rc = binding.load_library().fibar_readout_batch(None, None, None, 2, None, None, s)
        assert rc == FIBAR_EINVAL
        assert binding.fibar_readout_batch([], [], [], None, None, s) == 0
    finally:
        for f in a:
            f.close()


def test_memory_bytes_matches_the_allocation():
    from paper_2510_20071_gb300 import Fibar, memory_bytes
    for W, H, p in [(1280, 720, dict(blur_mode=1)), (346, 260, dict(blur_mode=0, max_pending=1 << 20))]:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        f = Fibar(W, H, **p)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        try:
            mb = f.memory_bytes()
            assert mb == memory_bytes(W, H, **p)
            delta = free0 - free1
            assert 0.9 * mb <= delta <= mb + (160 << 20), (W, H, mb, delta)
        finally:
            f.close()


def test_server_admits_by_memory():
    from paper_2510_20071_gb300.serving import Server, HANDLE_SLACK_BYTES
    from paper_2510_20071_gb300 import memory_bytes
    need = memory_bytes(64, 48, max_pending=1 << 16) + HANDLE_SLACK_BYTES
    srv = Server(budget=2 * need + need // 2)
    try:
        ids = [srv.admit(64, 48, max_pending=1 << 16) for _ in range(3)]
        assert ids[:2] == [0, 1] and ids[2] is None
        assert srv.stats()["refused"] == 1
        srv.release(ids[0])
        assert srv.admit(64, 48, max_pending=1 << 16) is not None
    finally:
        srv.close()

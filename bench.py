"""Benchmark: FIBAR events/s on one GB300 for the 1280x720 rotating/zooming Perlin stream.

Workload: 1280x720 sensor, 200 M events from the contrast-threshold simulator (C = 0.2)
over a rotating and zooming Perlin-noise texture with 2 % uniform noise events, seed 1,
pushed as device packets of 65,536 events with a read-out every 1,000,000 events.
One step = the pushes of one read-out interval plus the read-out (decode, sort, filter,
stale-pixel detector, masked-blur read-out into a device image).

Timed region: K steps after W warm-up steps, on the device with CUDA events, inputs
already in HBM; every step consumes a fresh 16 MB slice of the 3.2 GB stream (inputs
larger than L2).  `e2e` repeats the same steps through the C ABI from pinned HOST
buffers, with the host-to-device copies of the packets and the device-to-host copy of
each image inside the timed region.  `--impl reference` times the FP64 oracle on the
host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, H = 1280, 720
PACKET = 65_536
READ_EVERY = 1_000_000
STREAM_EVENTS = 200_000_000
CONFIG_NAME = "perlin_1280x720_200M"
METRIC = "events/s (M/s) on 1 GB300, % of HBM roofline; p50/p99 read-out latency"
UNIT = "Mevents/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per launch of the stage's kernel, from one ncu capture of the
# current kernel on this workload; a stage missing here has no capture of its current code.
# Cold-cache ncu capture (caches flushed before each launch), summed over the stage's kernels.
DRAM_TRAFFIC = {
    "s2": {"decode": 16.80e6, "sort": 8.03e6, "walk": 65.51e6, "det_counts": 41.01e6, "det_pass1": 16.97e6,
           "det_pass2": 11.67e6, "det_fix": 0.02e6, "readout": 11.07e6, "commit": 0.01e6},
    # S1 runs the same decode, sort and detector kernels on the same stream as S2
    "s1": {"decode": 16.80e6, "sort": 8.03e6, "walk": 86.84e6, "det_counts": 41.01e6, "det_pass1": 16.97e6,
           "det_pass2": 11.67e6, "det_fix": 0.02e6, "s1_blur": 159.54e6, "commit": 0.01e6},
}


MODE_PARAMS = {"s2": dict(spatial_filter=1, blur_mode=1), "s1": dict(spatial_filter=1, blur_mode=0),
               "nsf": dict(spatial_filter=0)}
MODE_NAMES = {"s2": "S2 masked-blur read-out", "s1": "S1 in-place blur (paper)", "nsf": "NSF (no spatial filter)"}
WORKLOAD = ("1280x720 rotating+zooming Perlin, 2% noise events, C=0.2, seed 1, 65,536-event device packets, "
            "read-out every 1,000,000 events")
PARITY_READOUTS = 20    # timed read-outs whose images are kept and compared with the oracle
PARITY_TOL = 1e-4       # absolute, per pixel, log brightness (C = 0.2)
ORACLE_SECONDS = 60.0   # bound on the oracle's replay of the warm-up and timed steps


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def whole_job(ms: float, events: float, world: int, device: str = "cuda"):
    """(max time over ranks in ms, events summed over ranks, whole-job Mevents/s): each
    rank times its own replica; the job takes as long as the slowest one."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, events], dtype=torch.float64, device=device)
    ms_t, ev_t = t[0:1].clone(), t[1:2].clone()
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(ev_t, op=dist.ReduceOp.SUM)
    ms_max, total = float(ms_t.item()), float(ev_t.item())
    return ms_max, total, total / (ms_max / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_plan(n_steps: int, t_col, packet: int = PACKET):
    """Per step: the (lo, hi) packets of the `packet`-event grid that end the step's
    read-out interval, and the read-out time (the interval's last time stamp)."""
    out, pushed = [], 0
    for s in range(n_steps):
        hi = (s + 1) * READ_EVERY
        pk = []
        while pushed < hi:
            pk.append((pushed, min(pushed + packet, len(t_col))))
            pushed += packet
        out.append((pk, int(t_col[hi - 1])))
    return out


class ClockSampler:
    """nvidia-smi samples (200 ms) while the GPU works."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(pw) if pw else None}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_stream(device, seed_offset=0):
    import eventsim
    cfg = dict(eventsim.CONFIGS[CONFIG_NAME])
    cfg["seed"] += seed_offset
    n = cfg.pop("n_events")
    return eventsim.simulate(cfg.pop("W"), cfg.pop("H"), n, device=device, **cfg)


def run_steps(f, ev, steps, out):
    for pk, t in steps:
        for lo, hi in pk:
            f.push(ev[lo:hi])
        f.readout(t, out)


BATCH_TICK_US = 1000


def run_batch(args, rank, world, local):
    """32 streams of mixed sensors (240x180, 346x260, 640x480, 1280x720) with mean event
    rates drawn log-uniformly from 0.5-20 Mev/s and Poisson read-out requests (100 Hz per
    stream), replayed as fast as the device allows: per 1 ms tick every stream's packet
    is pushed and the tick's requests are answered by concurrent batches (S2 read-out).
    A step is one tick; the timed region starts after a sweep that reads every stream out
    at the warm-up's end, and ends with every stream read out at its last event, so the
    events it applies are exactly those stamped after the warm-up."""
    import torch
    import torch.distributed as dist
    import eventsim
    from paper_2510_20071_gb300.serving import Server, latencies_ms

    t0 = time.time()
    seconds = args.batch_seconds
    streams = eventsim.mixed_streams(32, seconds, seed=11 + 1000 * rank, device=f"cuda:{local}")
    reqs = eventsim.request_times(32, seconds, rate_hz=100.0, seed=12 + 1000 * rank)
    torch.cuda.synchronize()
    n_ev = sum(s["events"].shape[0] for s in streams)
    log(f"[rank {rank}] simulated {len(streams)} streams, {n_ev} events in {time.time() - t0:.1f} s")
    sched = eventsim.serving_schedule(streams, reqs, tick_us=BATCH_TICK_US)
    # the first 40 % of the stream time is warm-up: every stream starts with an empty
    # queue, and the timed ticks measure streams whose queues have filled
    w = min(max(args.warmup, 2 * len(sched) // 5), len(sched) - 1)
    t_sweep = sched[w][0] - 1
    use_graph = args.batch_path == "graph"
    srv = Server(use_graph=use_graph)
    params = dict(c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=1)
    sids = [srv.admit(s["W"], s["H"], **params) for s in streams]
    if None in sids:
        raise RuntimeError("not enough device memory for the 32 streams")
    tuning = None
    if args.grid_share is not None:
        srv.set_grid_share({(s["W"], s["H"]): args.grid_share for s in streams})
        tuning = {"fixed_sms": args.grid_share}
    elif not args.no_autotune:
        # per sensor shape: the SM share with the most events/s when that shape's streams
        # are read out together, round after round without waiting (their read-outs
        # overlap as in serving), each at its shape's mean events per read-out (100 Hz)
        from paper_2510_20071_gb300.serving import GridTuner
        tuner = GridTuner(use_graph=use_graph)
        shapes = {}
        for s in streams:
            shapes.setdefault((s["W"], s["H"]), []).append(s["events"].shape[0] / seconds)
        t_tune = time.time()
        for (w_, h_), rates in shapes.items():
            tuner.tune(w_, h_, len(rates), int(sum(rates) / len(rates) / 100.0), **params)
        srv.set_grid_share(tuner.table)
        tuning = {"sms": {f"{w_}x{h_}": v for (w_, h_), v in tuner.table.items()},
                  "trials": {f"{w_}x{h_}": v for (w_, h_), v in tuner.trials.items()},
                  "seconds": round(time.time() - t_tune, 2)}
        log(f"[rank {rank}] grid shares {tuning['sms']} ({tuning['seconds']} s)")

    def tick(T, pushes, reads):
        # the tick's packet of every stream, in one library call
        srv.push_ranges([(sids[i], streams[i]["events"], lo, hi) for i, lo, hi in pushes])
        rs = [srv.request(sids[i], t) for i, t in reads]
        srv.serve()
        return rs

    for T, pushes, reads in sched[:w]:
        tick(T, pushes, reads)
    for i in range(len(streams)):
        srv.request(sids[i], t_sweep)
    srv.serve()
    st0 = srv.stats()
    stream = srv.stream
    timed = sched[w:]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    e0.record(stream)
    served = []
    for T, pushes, reads in timed:
        served += tick(T, pushes, reads)
    srv.join()  # group read-outs run on the streams' own CUDA streams
    e1.record(stream)
    host_ms = (time.perf_counter() - h0) * 1e3
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    time.sleep(0.3)
    clocks = sampler.stop()
    st1 = srv.stats()
    gstats = srv.group.stats() if srv.group is not None else None
    applied = st1["events_applied"] - st0["events_applied"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    lat = sorted(latencies_ms(served))
    expect = sum(int((s["events"][:, 1] > t_sweep).sum().item()) for s in streams)
    if applied != expect:
        raise RuntimeError(f"timed region applied {applied} events, expected {expect}")

    ms_max, _, value = whole_job(ms, float(applied), world)
    peak, peak_kind = load_peaks()
    px = sum(s["W"] * s["H"] for s in streams)
    img_bytes = 8.0 * sum(s["W"] * s["H"] * len([r for r in served if r.sid == sids[i]])
                          for i, s in enumerate(streams))
    alg = 16.0 * applied + img_bytes
    gbs = alg / (ms_max / 1e3) / 1e9

    def pct(p):
        return round(lat[min(len(lat) - 1, int(math.ceil(p / 100 * len(lat))) - 1)], 4) if lat else None

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": len(timed), "warmup": w, "ms_per_step": round(ms_max / max(len(timed), 1), 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded contrast-threshold simulator, 32 mixed streams)",
        "config": {"workload": f"32 streams: 8 each of 240x180, 346x260, 640x480, 1280x720; mean rates "
                               f"log-uniform 0.5-20 Mev/s; Poisson read-out requests at 100 Hz per stream; "
                               f"{seconds} s of stream time, 1 ms ticks; S2 read-out",
                   "streams": len(streams), "pixels": px, "events_timed": applied,
                   "requests_timed": len(served), "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: 32 streams' state and packets"},
        "roofline": {"bound": "hbm", "kernel": "whole batch (all stages)", "achieved": round(gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "traffic": None,
                     "peak_kind": peak_kind,
                     "alg_bytes": "16 B per event read + 8 B per pixel per image (L read, image written)"},
        "readout_latency_ms": {"p50": pct(50), "p99": pct(99), "max": pct(100), "samples": len(lat),
                               "what": "device time from the start of the request's batch (its first chain) to the request's image, queueing behind the stream's earlier read-outs included"},
        "host_ms": round(host_ms, 3),
        "grid_share_autotune": tuning,
        "serving_path": (f"group: each stream's read-out chain captured once as a CUDA graph, one graph launch "
                         f"per read-out on the stream's own CUDA stream ({gstats['graph_kernels']} kernel nodes in "
                         f"all, programmatic edges {'on' if gstats['programmatic_edges'] else 'off'}, "
                         f"{gstats['builds']} captures)" if gstats else "fibar_readout_batch: host launches on 16 streams"),
        "batches": st1["batches"] - st0["batches"],
        "clocks": clocks,
        "gpu_launches": launches,
    }
    srv.close()
    if rank == 0:
        print(json.dumps(result), flush=True)


PAN_CONFIG = "perlin_pan_1280x720_1B"
PAN_PACKETS = [8_192, 65_536, 1_048_576]


def run_pan(args, rank, world, local):
    """1280x720 Perlin noise panned in bursts (segments of 1-50 Mev/s), seed 2: the
    stream's first (W + K) x 1,000,000 events, read out every 1,000,000 events, pushed as
    device packets of 8,192, 65,536 and 1,048,576 events in turn (a fresh handle per size:
    W warm-up steps, then K timed steps).  The temporal filter's schedule is chosen per
    piece (auto); the line records how many pieces took the walk and the scan per size.
    `value` = events of all timed steps / their device time."""
    import torch
    import torch.distributed as dist
    import eventsim
    from paper_2510_20071_gb300 import Fibar

    n_steps = args.warmup + args.steps
    t0 = time.time()
    cfg = dict(eventsim.CONFIGS[PAN_CONFIG])
    cfg["seed"] += rank
    ev = eventsim.simulate(cfg.pop("W"), cfg.pop("H"), n_steps * READ_EVERY + max(PAN_PACKETS),
                           device=f"cuda:{local}", **{k: v for k, v in cfg.items() if k != "n_events"})
    torch.cuda.synchronize()
    log(f"[rank {rank}] simulated {ev.shape[0]} events in {time.time() - t0:.1f} s")
    t_col = ev[:, 1].cpu()
    params = dict(c_on=0.2, c_off=0.2, **MODE_PARAMS[args.mode])
    stream = torch.cuda.current_stream()
    out = torch.empty((H, W), dtype=torch.float32, device=ev.device)
    per_size, tot_ms, tot_ev, launches = {}, 0.0, 0, 0
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    check = None
    for packet in PAN_PACKETS:
        f = Fibar(W, H, stream=stream, **params)
        plan = step_plan(n_steps, t_col, packet)
        run_steps(f, ev, plan[:args.warmup], out)
        st0 = f.stats()
        timed = plan[args.warmup:]
        keep = packet == PACKET
        cmp_out = [torch.empty((H, W), dtype=torch.float32, device=ev.device)
                   for _ in range(min(len(timed), PARITY_READOUTS) if keep else 0)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, step in enumerate(timed):
            run_steps(f, ev, [step], cmp_out[i] if i < len(cmp_out) else out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        st = f.stats()
        applied = st["events_applied"] - st0["events_applied"]
        launches += st["kernel_launches"] - st0["kernel_launches"]
        if keep:
            check = (plan, f.state(), [o.cpu().numpy() for o in cmp_out])
        f.close()
        per_size[str(packet)] = {
            "value": round(applied / (ms / 1e3) / 1e6, 3), "ms_per_step": round(ms / len(timed), 5),
            "packets_per_step": len(timed[0][0]),
            "iir_walk_pieces": st["iir_walk_pieces"] - st0["iir_walk_pieces"],
            "iir_scan_pieces": st["iir_scan_pieces"] - st0["iir_scan_pieces"],
            "detector_fix_steps": st["detector_fix_steps"] - st0["detector_fix_steps"]}
        tot_ms += ms
        tot_ev += applied
    time.sleep(0.3)
    clocks = sampler.stop()
    ms_max, total, value = whole_job(tot_ms, float(tot_ev), world)
    peak, peak_kind = load_peaks()
    B_ev = 16.0 + 4.0 * W * H / READ_EVERY
    gbs = B_ev * total / (ms_max / 1e3) / 1e9
    n_timed = args.steps * len(PAN_PACKETS)
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / n_timed, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded contrast-threshold simulator)",
        "config": {"workload": "1280x720 Perlin noise panned in bursts (1-50 Mev/s segments), seed 2, "
                               "read-out every 1,000,000 events, device packets of 8,192 / 65,536 / "
                               "1,048,576 events (K timed steps each)",
                   "mode": MODE_NAMES[args.mode], "stream_events": int(ev.shape[0]),
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: each step reads a fresh 16 MB slice of the stream"},
        "per_packet_size": per_size,
        "roofline": {"bound": "hbm", "kernel": "whole step (all stages)", "achieved": round(gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "traffic": None,
                     "peak_kind": peak_kind, "alg_bytes_per_event": B_ev},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and check is not None:
        plan, gst, imgs = check
        result["cpu_baseline"], result["parity"] = run_cpu_baseline(ev, params, plan, args.warmup,
                                                                    plan[args.warmup:], imgs, gst)
        result["parity"]["packet"] = PACKET
    if rank == 0:
        print(json.dumps(result), flush=True)


FILL_TRAIN_SEEDS = list(range(101, 113))  # training streams (the benchmark stream, seed 1, is held out)
FILL_TRAIN_READOUTS = 6                   # frames per training stream (after 2 read-outs of start-up)
FILL_TRAIN_STEPS = 8000
FILL_BATCH = 512


def run_fill(args, rank, world, local):
    """Learned stale-pixel fill (blur_mode 2) on the benchmark stream.

    Training: 1280x720 Perlin streams of seeds 101-112 (6 read-outs each after 2 of queue
    start-up: 72 frames), FILL_TRAIN_STEPS Adam steps of FILL_BATCH 24x24 crops through
    fibar_fill_train_step.  Evaluation: RMSE over the stale pixels of 6 read-outs of the
    held-out benchmark stream (seed 1) against the simulator's log intensity in L units,
    for the learned fill, the Gaussian (S2) and no fill.  Timed region: K steps of the
    benchmark stream (as the headline) with the learned-fill read-out; `value` = events/s.
    The fill kernel's time per read-out comes from the stage pass, beside the S2 read-out's."""
    import numpy as np
    import torch
    import eventsim
    from paper_2510_20071_gb300 import Fibar
    from paper_2510_20071_gb300 import fill as FL

    t0 = time.time()
    train = FL.Frames.concat([FL.collect_frames(W, H, (2 + FILL_TRAIN_READOUTS) * READ_EVERY, seed=s)
                              for s in FILL_TRAIN_SEEDS])
    held = FL.collect_frames(W, H, 8 * READ_EVERY, seed=1 + rank)
    log(f"[rank {rank}] frames: {train.n} training, {held.n} held out ({time.time() - t0:.1f} s)")
    theta, train_s, hist = FL.train(train, FILL_TRAIN_STEPS, batch=FILL_BATCH, lr=3e-3, seed=rank, log_every=1000)
    quality = FL.evaluate(theta, held)
    del train, held

    n_stage = min(args.steps, 20)
    n_total = args.warmup + args.steps + n_stage
    cfg = dict(eventsim.CONFIGS[CONFIG_NAME])
    cfg["seed"] += rank
    ev = eventsim.simulate(cfg.pop("W"), cfg.pop("H"), n_total * READ_EVERY + PACKET, device=f"cuda:{local}",
                           **{k: v for k, v in cfg.items() if k != "n_events"})
    plan = step_plan(n_total, ev[:, 1].cpu())
    stream = torch.cuda.current_stream()
    out = torch.empty((H, W), dtype=torch.float32, device=ev.device)
    w0, w1 = args.warmup, args.warmup + args.steps

    def handle(mode):
        f = Fibar(W, H, stream=stream, c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=mode)
        if mode == 2:
            f.set_fill_weights(theta)
        return f

    f = handle(2)
    run_steps(f, ev, plan[:w0], out)
    st0 = f.stats()
    first = torch.empty_like(out)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i, step in enumerate(plan[w0:w1]):
        run_steps(f, ev, [step], first if i == 0 else out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    time.sleep(0.3)
    clocks = sampler.stop()
    st = f.stats()
    applied = st["events_applied"] - st0["events_applied"]
    launches = st["kernel_launches"] - st0["kernel_launches"]
    f.set_timing(True)
    f.stage_times(reset=True)
    run_steps(f, ev, plan[w1:], out)
    fill_stages = f.stage_times(reset=True)
    f.close()
    g = handle(1)
    run_steps(g, ev, plan[:w1], out)
    g.set_timing(True)
    g.stage_times(reset=True)
    run_steps(g, ev, plan[w1:], out)
    s2_stages = g.stage_times(reset=True)
    g.close()
    fill_ms = fill_stages["readout"] / max(fill_stages["calls"], 1)
    s2_ms = s2_stages["readout"] / max(s2_stages["calls"], 1)

    ms_max, total, value = whole_job(ms, float(applied), world)
    # all three 3x3 layers on the tensor cores: 2 x 9 x (2x16 + 16x16 + 16x1) FLOP per pixel
    # (the tiles' halo rows and columns, computed twice, are not counted)
    tc_flop = 2.0 * 9 * (2 * 16 + 16 * 16 + 16 * 1) * W * H
    tc_tflops = tc_flop / (fill_ms / 1e3) / 1e12
    peak_tf, peak_kind = load_tensor_peak()
    hbm, hbm_kind = load_peaks()
    fill_bytes = (4 + 8 + 4) * W * H   # L and last event read, image written
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, bf16 weights / fp32 accumulation (fill)",
        "data": "synthetic (seeded contrast-threshold simulator); fill trained on seeds 101-112, scored on seed 1",
        "config": {"workload": WORKLOAD, "mode": "learned stale-pixel fill (3x3 conv 2-16-16-1, blur_mode 2)",
                   "train_frames": FILL_TRAIN_READOUTS * len(FILL_TRAIN_SEEDS), "train_steps": FILL_TRAIN_STEPS,
                   "train_batch": FILL_BATCH, "crop": FL.CROP, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: each step reads a fresh 16 MB slice of the stream"},
        "fill": {"rmse_learned": round(quality["learned"], 5), "rmse_gaussian": round(quality["gaussian"], 5),
                 "rmse_no_fill": round(quality["none"], 5), "scored_pixels": quality["pixels"],
                 "what": "RMSE over stale pixels of 6 held-out read-outs against the simulator's log intensity "
                         "mapped into L units (per-frame least squares over the active pixels)",
                 "train_seconds": round(train_s, 3), "train_loss": hist,
                 "fill_readout_ms": round(fill_ms, 5), "gaussian_readout_ms": round(s2_ms, 5)},
        "roofline": {"bound": "tensor", "kernel": "k_fill (three 3x3 convs on tcgen05)", "achieved": round(tc_tflops, 2),
                     "peak": peak_tf, "unit": "TFLOP/s", "frac": round(tc_tflops / peak_tf, 5), "traffic": None,
                     "peak_kind": peak_kind,
                     "hbm_gbs": round(fill_bytes / (fill_ms / 1e3) / 1e9, 1), "hbm_peak": hbm,
                     "alg": "2 x 9 x 304 FLOP per pixel on the tensor cores; 16 B per pixel of HBM"},
        "stages_ms_per_step": {k: round(v / max(fill_stages["calls"], 1), 5) for k, v in fill_stages.items()
                               if k != "calls"},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["parity"] = fill_parity(ev, plan[:w0 + 1], theta, first.cpu().numpy())
    if rank == 0:
        print(json.dumps(result), flush=True)


def fill_parity(ev, plan, theta, gpu_img):
    """The first timed learned-fill image against the event oracle's state (same packets)
    passed through the fill oracle; bound as in the fill's parity tests (FP32 state of L
    propagated through the network, FP32 accumulation, rare BF16 rounding flips)."""
    import numpy as np
    import oracle
    from oracle import learned_fill as lf
    oracle.build()
    o = oracle.Oracle(W, H, c_on=0.2, c_off=0.2, spatial_filter=1, blur_mode=1)
    cpu = ev[:plan[-1][0][-1][1]].cpu()
    for pk, t in plan:
        for lo, hi in pk:
            o.push(cpu[lo:hi])
        o.readout(t)
    st = o.state()
    o.close()
    L = st["L"].reshape(H, W)
    age = lf.age_feature(st["k"], st["q"], st["last"]).reshape(H, W)
    stale = lf.stale_mask(st["h"], st["last"]).reshape(H, W)
    th = np.asarray(theta, dtype=np.float64)
    ref = np.where(stale, lf.forward(th, np.stack([L, age]))["y"], L)
    err = np.abs(gpu_img.astype(np.float64) - ref)
    return {"read_outs": 1, "max_abs_err": float(err.max()), "p999_abs_err": float(np.quantile(err, 0.999)),
            "frac_within_1e-3": float(np.mean(err <= 1e-3)), "pass": bool(np.mean(err <= 1e-3) >= 0.99),
            "what": "first timed learned-fill image against the FP64 event oracle's state through the FP64 "
                    "fill oracle"}


def load_tensor_peak():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


CALIB_EVENTS = 100_000_000


def run_calib(args, rank, world, local):
    """Relative contrast thresholds (fibar_relative_thresholds) of a 640x480 recording of
    100 M events (uniform random pixels and polarities, seeded): a step is one call over
    the whole recording, events resident on the device (16 B read per event; inputs far
    larger than L2).  e2e: the same call from pinned host memory (copies inside)."""
    import torch
    import torch.distributed as dist
    import eventsim
    from paper_2510_20071_gb300 import relative_thresholds

    W, H = 640, 480
    n_ev = args.calib_events
    ev = eventsim.random_events(W, H, n_ev, seed=21 + rank, p_on=0.52)
    dev = ev.to(f"cuda:{local}")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        relative_thresholds(dev, W, H)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        relative_thresholds(dev, W, H)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    time.sleep(0.3)
    clocks = sampler.stop()
    ms_max, total, _ = whole_job(ms, float(n_ev) * args.steps, world)
    per = ms_max / args.steps
    value = total / args.steps / (per / 1e3) / 1e6
    # e2e: pinned host events through the host path of the same call
    pinned = ev.pin_memory()
    n_e2e = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        relative_thresholds(pinned, W, H)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    peak, peak_kind = load_peaks()
    alg = 16.0 * n_ev + 12.0 * W * H + 8.0 * W * H
    gbs = alg / (per / 1e3) / 1e9
    result = {
        "metric": "calibration events/s (M/s) on 1 GB300, % of HBM roofline", "value": round(value, 3),
        "unit": "Mevents/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(per, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 counts, f32 thresholds", "data": "synthetic (uniform random 640x480 events, seeded)",
        "config": {"workload": f"relative contrast thresholds of a 640x480 recording, {n_ev} events",
                   "l2": f"inputs larger than L2: {16 * n_ev / 1e9:.2f} GB of records per step"},
        "roofline": {"bound": "hbm", "kernel": "k_calib_count + k_calib_finish", "achieved": round(gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "traffic": None,
                     "peak_kind": peak_kind,
                     "alg_bytes": "16 B per record read, 8 B per pixel of counts, 12 B per pixel written"},
        "e2e": {"value": round(n_ev / (e2e_ms / 1e3) / 1e6, 3), "unit": "Mevents/s",
                "h2d_bytes_per_step": 16 * n_ev, "d2h_bytes_per_step": 12 * W * H},
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--mode", default="s2", choices=["s2", "s1", "nsf"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stream-events", type=int, default=None,
                    help="simulate a shorter stream (profiling runs); default: the 200 M workload")
    ap.add_argument("--workload", default="stream", choices=["stream", "pan", "fill", "batch32", "calib"],
                    help="stream: one 1280x720 stream (the headline); pan: the bursty 1280x720 pan "
                         "stream at three packet sizes; fill: the learned stale-pixel fill; batch32: 32 mixed streams served in concurrent "
                         "batches; calib: relative thresholds of a 640x480 recording")
    ap.add_argument("--batch-seconds", type=float, default=0.2,
                    help="batch32: stream time simulated per stream")
    ap.add_argument("--grid-share", type=int, default=None,
                    help="batch32: SMs every stream's grids are sized for (default: autotuned per shape)")
    ap.add_argument("--no-autotune", action="store_true", help="batch32: whole-device grids for every stream")
    ap.add_argument("--batch-path", default="graph", choices=["graph", "streams"],
                    help="batch32: group read-outs (one captured graph per stream, launched on the "
                         "stream's own CUDA stream), or fibar_readout_batch's host launches")
    ap.add_argument("--calib-events", type=int, default=100_000_000,
                    help="calib: records in the recording (profiling runs use fewer)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    if args.workload == "batch32":
        # hardware work queues for the streams' own CUDA streams (read by CUDA when the
        # context is created): measured 1849 / 2003 / 1972-1995 Mev/s with 8 / 16 / 32,
        # p99 latency 2.6 / 4.0 / 6.5 ms
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "16")
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if args.workload == "batch32":
        return run_batch(args, rank, world, local)
    if args.workload == "calib":
        return run_calib(args, rank, world, local)
    if args.workload == "pan":
        return run_pan(args, rank, world, local)
    if args.workload == "fill":
        return run_fill(args, rank, world, local)
    from paper_2510_20071_gb300 import Fibar

    n_lat = min(args.steps, 50)     # read-out latency pass
    n_stage = min(args.steps, 20)   # per-stage timing pass
    n_total = args.warmup + args.steps + n_lat + n_stage
    need = n_total * READ_EVERY
    stream_events = max(args.stream_events or STREAM_EVENTS, need + PACKET)
    t0 = time.time()
    import eventsim
    cfg = dict(eventsim.CONFIGS[CONFIG_NAME])
    cfg["seed"] += rank
    cfg["n_events"] = stream_events
    ev = eventsim.simulate(cfg.pop("W"), cfg.pop("H"), cfg.pop("n_events"), device=f"cuda:{local}", **cfg)
    torch.cuda.synchronize()
    log(f"[rank {rank}] simulated {ev.shape[0]} events in {time.time() - t0:.1f} s")

    params = dict(c_on=0.2, c_off=0.2, **MODE_PARAMS[args.mode])
    stream = torch.cuda.current_stream()
    f = Fibar(W, H, stream=stream, **params)
    plan = step_plan(n_total, ev[:, 1].cpu())
    out = torch.empty((H, W), dtype=torch.float32, device=ev.device)
    w0, w1 = args.warmup, args.warmup + args.steps
    run_steps(f, ev, plan[:w0], out)
    timed = plan[w0:w1]
    det0 = f.stats()
    launches0 = det0["kernel_launches"]
    applied0 = det0["events_applied"]

    # timed region: K steps, no instrumentation between the kernels
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.4)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # the first PARITY_READOUTS timed steps write their images to buffers of their own
    # (checked against the oracle after the run); the others reuse one buffer
    n_cmp = min(len(timed), PARITY_READOUTS)
    cmp_out = [torch.empty((H, W), dtype=torch.float32, device=ev.device) for _ in range(n_cmp)]
    torch.cuda.synchronize()
    e0.record(stream)
    for i, step in enumerate(timed):
        run_steps(f, ev, [step], cmp_out[i] if i < n_cmp else out)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    time.sleep(0.3)
    clocks = sampler.stop()
    st = f.stats()
    applied = st["events_applied"] - applied0
    launches = st["kernel_launches"] - launches0
    gpu_state = f.state()  # after the last timed step, for the oracle check
    gpu_imgs = [o.cpu().numpy() for o in cmp_out]
    del cmp_out

    # read-out latency: one step per event pair (all of a step's work runs in its read-out)
    lat = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_lat)]
    for (a, b), step in zip(evs, plan[w1:w1 + n_lat]):
        a.record(stream)
        run_steps(f, ev, [step], out)
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in evs)

    # per-stage CUDA-event times (events between the pipeline's kernels)
    f.stage_times(reset=True)
    f.set_timing(True)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    run_steps(f, ev, plan[w1 + n_lat:w1 + n_lat + n_stage], out)
    s1.record(stream)
    torch.cuda.synchronize()
    stages = f.stage_times(reset=True)
    f.set_timing(False)
    stage_pass_ms = s0.elapsed_time(s1) / max(n_stage, 1)

    # the other spatial-filter modes on the same stream and steps (a fresh handle each):
    # the paper's in-place blur (S1) and no spatial filter (NSF), timed like `value`
    modes = {}
    if args.mode == "s2":
        k_modes = min(args.steps, 20)
        for m in ("s1", "nsf"):
            fm = Fibar(W, H, stream=stream, c_on=0.2, c_off=0.2, **MODE_PARAMS[m])
            run_steps(fm, ev, plan[:w0], out)
            a0 = fm.stats()["events_applied"]
            torch.cuda.synchronize()
            m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            run_steps(fm, ev, plan[w0:w0 + k_modes], out)
            m1.record(stream)
            torch.cuda.synchronize()
            mms = m0.elapsed_time(m1)
            ma = fm.stats()["events_applied"] - a0
            modes[m] = {"name": MODE_NAMES[m], "value": round(ma / (mms / 1e3) / 1e6, 3),
                        "ms_per_step": round(mms / k_modes, 5), "steps": k_modes, "unit": UNIT}
            fm.close()

    ms_max, total_events, value = whole_job(ms, float(applied), world)  # Mevents/s, whole job

    # roofline of the dominant kernel stage, from its CUDA-event time in the stage pass
    peak, peak_kind = load_peaks()
    steps = len(timed)
    per_step_events = applied / steps
    B_ev = 16.0 + 4.0 * W * H / READ_EVERY
    stage_ms = {k: v for k, v in stages.items() if k != "calls"}
    dom = max(stage_ms, key=stage_ms.get)
    # algorithmic bytes per stage launch: decode reads the 16 B records; the read-out
    # writes the W*H float image (S2 also reads L: 4 B/px); other stages operate on
    # L2-resident intermediates and have no compulsory HBM bytes of their own, so the
    # whole step's algorithmic bytes are charged to them.
    alg_bytes = {"decode": 16.0 * per_step_events, "readout": 8.0 * W * H}
    bytes_per_launch = alg_bytes.get(dom, B_ev * per_step_events)
    dom_ms = stage_ms[dom] / max(stages["calls"], 1)
    achieved = bytes_per_launch / (dom_ms / 1e3) / 1e9
    whole_gbs = B_ev * total_events / (ms_max / 1e3) / 1e9

    def pct(p):
        return round(lat[min(len(lat) - 1, int(math.ceil(p / 100 * len(lat))) - 1)], 4) if lat else None

    result = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded contrast-threshold simulator)",
        "config": {"workload": WORKLOAD,
                   "mode": MODE_NAMES[args.mode],
                   "stream_events": int(ev.shape[0]), "events_per_step": int(per_step_events),
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2: each step reads a fresh 16 MB slice of the 3.2 GB stream"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": DRAM_TRAFFIC.get(args.mode, {}).get(dom),
                     "peak_kind": peak_kind,
                     "whole_step_gbs": round(whole_gbs, 1),
                     "whole_step_frac": round(whole_gbs / peak, 4),
                     "alg_bytes_per_event": B_ev},
        "readout_latency_ms": {"p50": pct(50), "p99": pct(99), "max": pct(100), "samples": len(lat),
                               "what": "device time of one read-out (1 M pending events + image)"},
        "modes": modes or None,
        "stages_ms_per_step": {k: round(v / max(stages["calls"], 1), 5) for k, v in stage_ms.items()},
        "stage_pass_ms_per_step": round(stage_pass_ms, 5),
        "clocks": clocks,
        "gpu_launches": int(launches),
        "detector": {k: st[k] - det0[k] for k in ["detector_fixups", "detector_unmerged",
                                                   "detector_pass2_steps", "detector_fix_steps", "s1_blurs",
                                                   "detector_big_pops", "detector_ring_misses",
                                                   "detector_recenters"]},
    }

    if not args.no_e2e:
        result["e2e"] = run_e2e(args, ev, plan[:w1], params, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"], result["parity"] = run_cpu_baseline(ev, params, plan, w0, timed, gpu_imgs,
                                                                    gpu_state)
    f.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, ev, plan, params, torch):
    """Same steps through the C ABI from pinned host memory, every image read back to the
    host: each step pushes its packets (host-to-device copy on the library's copy stream)
    and queues its read-out with the image's device-to-host copy; the host waits for the
    previous step's image before it reuses that image's buffer, so one step's copies
    overlap the other's pipeline.  The timed region ends when the last image is on the
    host."""
    from paper_2510_20071_gb300 import Fibar
    stream = torch.cuda.current_stream()
    lo_all = plan[args.warmup][0][0][0]
    hi_all = plan[-1][0][-1][1]
    host = torch.empty((hi_all - lo_all, 2), dtype=torch.int64).pin_memory()
    host.copy_(ev[lo_all:hi_all])
    warm = torch.empty((plan[args.warmup - 1][0][-1][1], 2), dtype=torch.int64).pin_memory()
    warm.copy_(ev[: warm.shape[0]])
    out = torch.empty((H, W), dtype=torch.float32).pin_memory()
    f = Fibar(W, H, stream=stream, **params)
    for pk, t in plan[: args.warmup]:
        for lo, hi in pk:
            f.push(warm[lo:hi])
        f.readout(t, out)
    outs = [out, torch.empty((H, W), dtype=torch.float32).pin_memory()]
    torch.cuda.synchronize()
    applied0 = f.stats()["events_applied"]
    t0 = time.perf_counter()
    done = []
    for i, (pk, t) in enumerate(plan[args.warmup:]):
        # the step's packets in one call (adjacent packets: one host-to-device copy, on the
        # library's copy stream: it overlaps the previous step's read-out)
        f.push_many([host[lo - lo_all:hi - lo_all] for lo, hi in pk])
        f.readout_host_async(t, outs[i % 2])
        ev = torch.cuda.Event()
        ev.record(stream)
        done.append(ev)
        if i >= 1:
            done[i - 1].synchronize()  # the previous step's image is on the host
    f.wait()
    dt = time.perf_counter() - t0
    applied = f.stats()["events_applied"] - applied0
    f.close()
    steps = len(plan) - args.warmup
    n = sum(hi - lo for pk, _ in plan[args.warmup:] for lo, hi in pk)
    return {"value": round(applied / dt / 1e6, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(16 * n / steps), "d2h_bytes_per_step": int(4 * W * H),
            "ms_per_step": round(dt * 1e3 / steps, 4)}


def run_cpu_baseline(ev, params, plan, w0, timed, gpu_imgs, gpu_state):
    """The FP64 oracle, single-threaded, replaying the GPU run's own packets and read-outs:
    the warm-up steps, then the timed steps (bounded by ORACLE_SECONDS).  Its throughput is
    the CPU baseline; its images of the first timed read-outs and its state after the last
    timed step are compared with the GPU's (images within PARITY_TOL, integer state
    bit-exact)."""
    import numpy as np
    import oracle
    oracle.build()
    o = oracle.Oracle(W, H, **params)
    n_steps = w0 + len(timed)
    hi_all = plan[n_steps - 1][0][-1][1]
    cpu = ev[:hi_all].cpu()
    busy, worst, compared, reached = 0.0, 0.0, 0, 0
    for s_i, (pk, t) in enumerate(plan[:n_steps]):
        t0 = time.perf_counter()
        for lo, hi in pk:
            o.push(cpu[lo:hi])
        img = o.readout(t)
        busy += time.perf_counter() - t0
        reached = s_i + 1
        j = s_i - w0
        if 0 <= j < len(gpu_imgs):
            worst = max(worst, float(np.abs(img - gpu_imgs[j].astype(np.float64)).max()))
            compared += 1
        if busy > ORACLE_SECONDS and j >= len(gpu_imgs) - 1:
            break
    ost = o.state()
    applied = ost["k"]
    int_equal = None
    state_err = None
    if reached == n_steps:
        keys = ["k", "h", "q", "q_targ", "n_ap", "n_at"] if params.get("spatial_filter", 1) else ["k"]
        int_equal = all(int(gpu_state[k]) == int(ost[k]) for k in keys)
        int_equal = int_equal and bool(np.array_equal(gpu_state["last_idx"], ost["last"].astype(np.uint64)))
        if params.get("spatial_filter", 1):
            int_equal = int_equal and bool(np.array_equal(gpu_state["cnt"], ost["cnt"]))
        state_err = max(float(np.abs(gpu_state["L"] - ost["L"]).max()),
                        float(np.abs(gpu_state["pbar"] - ost["pbar"]).max()))
    o.close()
    ok = compared == len(gpu_imgs) and worst <= PARITY_TOL and int_equal is not False and \
        (state_err is None or state_err <= PARITY_TOL)
    baseline = {"value": round(applied / busy / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the run's first {reached} read-out intervals ({applied} events: {w0} warm-up and "
                          f"{reached - w0} timed steps) with the same packets and read-out times, FP64 "
                          f"event-by-event, one thread"}
    parity = {"read_outs": compared, "timed_steps_compared": [0, compared], "max_abs_err": worst,
              "tol": PARITY_TOL, "int_state_equal": int_equal,
              "state_after_step": n_steps if reached == n_steps else None,
              "state_max_abs_err": state_err, "pass": bool(ok),
              "what": "GPU images of the first timed read-outs and the GPU state after the last timed step "
                      "against the FP64 oracle replaying the same packets (k, h, q, q_targ, N_ap, N_at, "
                      "per-pixel queued counts and last event index bit-exact; images, L, p_bar within tol)"}
    return baseline, parity


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same workload / metric / unit and
    mode.  Each step pushes a bounded sample of the stream (the whole read-out interval
    of 1,000,000 events when K <= 20, else 20/K of it) as 65,536-event packets and reads
    out at its last time stamp."""
    if rank != 0:
        return 0
    import torch
    import oracle
    import eventsim
    oracle.build()
    mode_params = MODE_PARAMS[args.mode]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    per_step = max(1, min(READ_EVERY, int(READ_EVERY * 20 / max(args.steps, 1))))
    n = (args.warmup + args.steps) * per_step
    cfg = dict(eventsim.CONFIGS[CONFIG_NAME])
    cfg["n_events"] = STREAM_EVENTS if dev == "cuda" else n
    ev = eventsim.simulate(cfg.pop("W"), cfg.pop("H"), cfg.pop("n_events"), device=dev, **cfg)[:n].cpu()
    t_col = ev[:, 1]
    o = oracle.Oracle(W, H, c_on=0.2, c_off=0.2, **mode_params)

    def step(pos):
        for lo in range(pos, pos + per_step, PACKET):
            o.push(ev[lo:min(lo + PACKET, pos + per_step)])
        o.readout(int(t_col[pos + per_step - 1]))

    pos = 0
    for _ in range(args.warmup):
        step(pos)
        pos += per_step
    t0 = time.perf_counter()
    applied0 = o.state()["k"]
    for _ in range(args.steps):
        step(pos)
        pos += per_step
    dt = time.perf_counter() - t0
    done = o.state()["k"] - applied0
    value = done / dt / 1e6
    res = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded contrast-threshold simulator)", "impl": "reference",
           "config": {"workload": WORKLOAD, "mode": MODE_NAMES[args.mode], "events_per_step": per_step},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{per_step} events per step of the same stream, FP64, one thread"},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main() or 0)

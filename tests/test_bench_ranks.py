"""The benchmark's whole-job numbers over replicas (one stream per rank, no collective on
the data path): two gloo ranks on the CPU, each with its own time and event count."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]
    events = [4.0e8, 5.0e8][rank]
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    out[rank] = bench.whole_job(ms, events, world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_is_max_time_and_summed_events():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork: the parent may hold threads
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        got = dict(out)
    for rank in range(world):
        ms_max, total, value = got[rank]
        assert ms_max == 150.0 and total == 9.0e8
        assert value == pytest.approx(9.0e8 / 0.150 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.whole_job(10.0, 1.0e6, 1, device="cpu") == (10.0, 1.0e6, pytest.approx(100.0))

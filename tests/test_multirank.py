"""Host logic of bench.py for N > 1 ranks, run as two gloo ranks on the CPU:
the job's time is the slowest rank's and the job's throughput counts every
rank's replica (weak scaling, no data-path collective)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, "cpu")
    value = bench.job_value(1000 * 3 * 10, ms_max, world)
    ws, r, local = bench._dist_env()
    out[rank] = (ms_max, value, ws, r, local)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_time_and_whole_job_value():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms_max, value, ws, r, local = res[rank]
        assert ms_max == 15.0
        assert value == pytest.approx(1000 * 3 * 10 * 2 / 0.015)
        assert (ws, r, local) == (2, rank, rank)


def test_single_rank_needs_no_process_group():
    import bench
    assert not dist.is_initialized()
    assert bench.max_over_ranks(12.5, "cpu") == 12.5
    assert bench.job_value(300, 10.0, 1) == pytest.approx(30000.0)

"""The multi-GPU form is replicas (the single-box path does not shard): each rank evaluates its
own box and the job's throughput uses the slowest rank's time.  This host-side logic of bench.py
runs here on two gloo ranks on the CPU."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 30.0][rank]
    m = bench.max_over_ranks(ms, "cpu")
    v = bench.job_throughput(1000, 4, world, m)
    out[rank] = (m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 30.0
    assert res[0][1] == pytest.approx(1000 * 4 * 2 / 0.030)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.0, "cpu") == 7.0
    assert bench.job_throughput(10, 2, 1, 4.0) == pytest.approx(5000.0)

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


def test_partition_balances_uneven_boxes():
    from paper_2003_13218_gb300 import boxes, shard
    wins = [boxes.lambda_windows(64, seed=0)[i][0].N for i in range(64)]
    costs = [shard.box_cost(n) for n in wins]
    for world in (1, 2, 3, 8):
        parts = shard.partition_boxes(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT keeps the heaviest rank within the largest single box of the mean
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.partition_boxes([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    from paper_2003_13218_gb300 import shard
    costs = [3.0, 9.0, 1.0, 4.0, 7.0, 2.0, 8.0]
    mine = shard.partition_boxes(costs, world)[rank]
    # each rank "evaluates" its boxes: a value that identifies the box and the rank that computed it
    local = {"e_total": np.array([-1000.0 * i - 0.5 for i in mine]), "rank": np.array([float(rank)] * len(mine))}
    res = shard.gather_box_results(local, mine, len(costs))
    out[rank] = None if res is None else {k: v.tolist() for k, v in res.items()}
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_batch_gathers_every_box_in_order():
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] is None
    r0 = res[0]
    assert r0["e_total"] == [-1000.0 * i - 0.5 for i in range(7)]
    # boxes 1 (9), 6 (8) ... alternate by load; both ranks contributed
    assert set(r0["rank"]) == {0.0, 1.0}

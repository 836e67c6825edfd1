"""Host logic of the N > 1 bench path on CPU: two gloo ranks, each with its
own timing, aggregate to the slowest rank; the reference arm prints on
rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world)
    val = bench.whole_job_gcups(1e12, 4, mx[0], world)
    dist.barrier()
    out[rank] = (mx, val)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        mx, val = out[r]
        assert mx == [11.0, 5.0]
        assert val == pytest.approx(2 * 1e12 * 4 / (11.0 / 1e3) / 1e9)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.whole_job_gcups(1e9, 1, 1000.0, 1) == pytest.approx(1.0)


def test_reference_arm_is_rank0_only(capsys):
    import bench

    class A:
        n, steps, warmup = 8, 1, 0

    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""

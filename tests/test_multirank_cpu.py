"""The replica (weak-scaling) path of bench.py on two gloo ranks, on CPU.

The path has no data-path collective: each rank evaluates its own copy of the
workload; the bench takes the slowest rank's time and counts every rank's
atoms.  This checks that reduction with world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 250.0][rank]
    dist.barrier()
    worst = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.replica_throughput(1000, 10, world, worst)
    out[rank] = (worst, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_slowest_rank_and_count_all_atoms():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0][0] == 250.0 and out[1][0] == 250.0
    assert out[0][1] == pytest.approx(2 * 1000 * 10 / 0.25)

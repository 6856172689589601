"""The N > 1 path of bench.py (independent replicas, one per GPU): the slowest
rank's time sets the whole-job throughput.  Run as two gloo ranks on CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_seconds = [0.5, 2.0][rank]
    slowest = bench.max_over_ranks(per_rank_seconds)
    value = bench.job_throughput(1.0e9, slowest, world)
    out[rank] = (slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        slowest, value = out[r]
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1.0e9 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0

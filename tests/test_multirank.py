"""The N > 1 path of bench.py (one replica per rank, whole-job throughput over the slowest
rank) on CPU with the gloo backend, world size 2."""
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
    seconds = 2.0 if rank == 0 else 3.0      # the slower rank sets the job time
    slowest, value = bench.aggregate(seconds, 600.0, world, dist, torch.device("cpu"))
    out[rank] = (slowest, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, value = res[rank]
        assert slowest == 3.0
        assert value == 600.0 * 2 / 3.0


def test_single_rank_uses_no_collective():
    import bench
    slowest, value = bench.aggregate(4.0, 100.0, 1)
    assert slowest == 4.0 and value == 25.0

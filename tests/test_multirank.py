"""The N > 1 paths on CPU with the gloo backend, world size 2: bench.py's replicas (whole-job
throughput over the slowest rank), and the split of independent (medium, species) units over
ranks with one gather of the Z/D series at the end (paper_1303_2470_gb300.shard; the units
are run by the oracle here, so no GPU is needed)."""
import os
import socket

import numpy as np
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


# ---- species / media split over ranks (paper_1303_2470_gb300.shard) ------------------------
def _media():
    from paper_1303_2470_gb300 import media
    out = []
    for j, shape in enumerate(((9, 10, 11), (8, 12, 7))):
        solid, _ = media.random_spheres(shape, 2, 0.6, seed=20 + j)
        u = media.drift_flow(solid, 0.005, 0.004, seed=30 + j)
        out.append((solid, u, media.species(3, seed=40 + j, D_b=(0.03, 0.1))))
    return out


def _oracle_runner(medium, species, steps):
    import oracle
    solid, u, (Db, ka, kd) = medium
    res = {}
    for s in species:
        r = oracle.run(oracle.Problem(solid, u, Db[s], ka[s], kd[s]), g=0, nsteps=steps)
        res[s] = (r.Z, r.D)
    return res


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1303_2470_gb300 import shard
    meds = _media()
    units = [(m, s) for m in range(len(meds)) for s in range(3)]
    got = shard.run_sharded(meds, units, 40, _oracle_runner, rank=rank, world=world, dist=dist)
    out[rank] = {f"{k[0]},{k[1]}": (v[0].tolist(), v[1].tolist()) for k, v in got.items()}
    dist.barrier()
    dist.destroy_process_group()


def test_units_are_split_in_balanced_contiguous_runs():
    from paper_1303_2470_gb300 import shard
    units = list(range(11))
    for world in (1, 2, 3, 4, 11, 16):
        parts = shard.split_units(units, world)
        assert len(parts) == world and sum(parts, []) == units
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1


def test_two_ranks_gather_the_series_of_a_single_rank_run():
    """Two gloo ranks each run half of the (medium, species) units and all-gather the Z(t),
    D(t) series: both ranks hold every unit's series, equal to a one-rank run of all units."""
    from paper_1303_2470_gb300 import shard
    meds = _media()
    units = [(m, s) for m in range(len(meds)) for s in range(3)]
    ref = shard.run_sharded(meds, units, 40, _oracle_runner)
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert sorted(res[rank]) == sorted(f"{a},{b}" for a, b in units)
        for (a, b), (z, d) in ref.items():
            zz, dd = res[rank][f"{a},{b}"]
            assert np.array_equal(np.asarray(zz), z) and np.array_equal(np.asarray(dd), d)


def test_gather_refuses_a_unit_run_twice():
    from paper_1303_2470_gb300 import shard

    class FakeDist:
        def all_gather_object(self, parts, obj):
            parts[0] = obj
            parts[1] = obj
    with pytest.raises(ValueError, match="two ranks"):
        shard.gather_series({(0, 0): (np.zeros(3), np.zeros(3))}, FakeDist(), 2)

"""The benchmark's multi-GPU path on CPU: two gloo ranks (one process each)
check the weak-scaling bookkeeping -- each rank maps its own seeded cube, the
job's step time is the slowest rank's (max over ranks), and the whole-job
value counts every rank's seeds. No data-path collective exists: the lines of
one rank never need another rank's data."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    B, grid, u, v = bench.monopole24_inputs(r, cube=(16, 12, 8))
    # a made-up per-rank step time: the slower rank sets the job's time
    ms_local = 2.0 + r
    ms, value = bench.job_rate(ms_local, 1000, dist, "cpu")
    out[r] = (ws, local, float(B.sum()), ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        ws, local, bsum, ms, value = res[r]
        assert ws == world and local == r
        assert ms == 3.0  # the max over ranks
        assert value == pytest.approx(1000 * world / 3e-3)
    # each rank traced its own cube
    assert res[0][2] != res[1][2]


def test_single_process_rate():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    ms, value = bench.job_rate(4.0, 500)
    assert ms == 4.0 and value == pytest.approx(500 / 4e-3)
    assert np.isfinite(value)

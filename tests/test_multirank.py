"""The multi-process path of bench.py on CPU ranks (gloo, world size 2).

Each rank runs its own replica (no data-path collective); the step time is the
maximum over ranks and the job's value counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                       # the second replica is slower
    got = bench.max_over_ranks(ms, dist, "cpu")
    val = bench.job_value(1e9, world, got)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, "r%d" % rank), "w") as f:
        f.write("%r %r" % (got, val))


def test_two_gloo_ranks_take_the_slowest_replica(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got, val = (float(x) for x in open(tmp_path / ("r%d" % r)).read().split())
        assert got == 15.0
        assert abs(val - 2 * 1e9 / 0.015 / 1e9) < 1e-9


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(2e9, 1, 1000.0) == 2.0

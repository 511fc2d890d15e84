"""The multi-GPU path of bench.py on CPU: two gloo ranks (one process each), as torchrun
launches them.  Each rank times its own replica; the job's time is the maximum over the
ranks (a barrier brackets the timed region) and the value counts every rank's units."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    total, value = bench.job_throughput(local_ms, units_per_rank=1000, steps=4, world=world, device="cpu")
    dist.barrier()
    out[rank] = (total, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        total, value = res[r]
        assert total == 200.0                          # max over ranks, seen by every rank
        assert value == pytest.approx(1000 * 4 * world / 0.2)


def test_single_rank_needs_no_process_group():
    import bench
    total, value = bench.job_throughput(50.0, units_per_rank=10, steps=5, world=1)
    assert total == 50.0 and value == pytest.approx(10 * 5 / 0.05)

"""The N > 1 path of the benchmark is replicas only (the factorization does not
shard across GPUs): every rank runs its own copy of the workload, and the job's
time is the slowest rank's.  Two CPU processes over gloo check the aggregation
the benchmark uses (max over ranks, whole-job value = ranks x units / that
time) and that a barrier-separated step count agrees across ranks."""
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


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = [100.0, 150.0][rank]                   # rank 1 is the slow replica
        ms = bench.max_over_ranks(ms_local, world, "cpu")
        units = 3 * 4096 * 16
        value = bench.job_value(units, world, ms)
        steps = torch.tensor([3.0])
        dist.all_reduce(steps, op=dist.ReduceOp.MAX)
        dist.barrier()
        out[rank] = (ms, value, float(steps.item()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as manager:
        out = manager.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        ms, value, steps = res[r]
        assert ms == 150.0                                 # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 3 * 4096 * 16 / 0.150)
        assert steps == 3.0


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.job_value(1000, 1, 500.0) == pytest.approx(2000.0)

"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

Every GPU runs an independent replica of the workload (weak scaling, no
data-path collective); the only cross-rank steps are the barrier around the
timed region and the reduction of the timing and unit counts, where the job
time is the slowest rank's and the value counts every rank's units.
"""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        rmax, rsum = bench.reducers(dist, "cpu")
        # rank r ran 10 + r units in 1.0 + 0.5 r seconds
        value, t, units = bench.aggregate(1.0 + 0.5 * rank, 10 + rank, ws, rmax, rsum)
        dist.barrier()
        q.put((rank, ws, r, local, value, t, units))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_weak_scaling_aggregation_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total_units = sum(10 + r for r in range(world))
    t_max = 1.0 + 0.5 * (world - 1)
    for rank, ws, r, local, value, t, units in res:
        assert (ws, r, local) == (world, rank, rank)
        assert units == total_units
        assert t == pytest.approx(t_max)
        assert value == pytest.approx(total_units / t_max)


def test_single_rank_aggregation_needs_no_process_group():
    import bench

    rmax, rsum = bench.reducers(None, "cpu")
    value, t, units = bench.aggregate(2.0, 8, 1, rmax, rsum)
    assert (value, t, units) == (4.0, 2.0, 8)


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    """Under torchrun the CPU-oracle reference arm is timed by rank 0 alone;
    the other ranks exit without work or output."""
    import sys

    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.main()
    assert capsys.readouterr().out == ""

"""The N > 1 path of bench.py (independent replicas, no data-path collective) on two gloo ranks
on the CPU: the slowest rank's time sets the step, the whole-job value counts every rank's
blocks, and the reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.rank_info()
    t_ms = 100.0 + 10.0 * rank                       # rank 1 is the slower replica
    dist.barrier()
    t_max = bench.max_over_ranks(t_ms, dist, "cpu")
    per_step, value = bench.job_ms_per_block(t_max, steps, w)
    out[rank] = (r, w, loc, t_max, per_step, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_job_value():
    world, steps = 2, 5
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, port, steps, out), nprocs=world, join=True)
    for rank in range(world):
        r, w, loc, t_max, per_step, value = out[rank]
        assert (r, w, loc) == (rank, world, rank)
        assert t_max == 110.0                      # every rank sees the slowest replica
        assert per_step == 110.0 / steps
        assert value == 110.0 / (steps * world)    # blocks of both replicas in that time


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""

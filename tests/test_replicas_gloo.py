"""The multi-GPU path is replicas only: N ranks run independent instances, the step time is the
maximum over ranks and the throughput counts every rank's work. Exercised here with two gloo ranks
on the CPU (no GPU, no NCCL)."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 10.0 + 5.0 * rank            # the slower rank sets the pace
    ms, value = bench.replica_aggregate(local_ms, 1e9, world, allreduce_max)
    w, r, _ = bench._dist()
    out[rank] = (ms, value, w, r)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_total_units():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        ms, value, w, r = out[rank]
        assert (w, r) == (world, rank)
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(2 * 1e9 / 0.015)


def test_single_rank_needs_no_reduction():
    ms, value = bench.replica_aggregate(12.5, 4e9, 1, None)
    assert ms == 12.5 and value == pytest.approx(4e9 / 0.0125)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""

"""The multi-GPU path of the benchmark (independent replicas, max-over-ranks
timing) on CPU process groups: world size 2, gloo backend."""
import os
import socket

import pytest

from paper_1012_3911_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # each rank "times" its own replica; the slowest one sets the job time
        local_ms = 100.0 + 25.0 * rank
        job_ms = replicas.max_over_ranks(local_ms, dist)
        dist.barrier()
        value = replicas.job_throughput(1000, 50, 3, world, job_ms)
        out.put((rank, job_ms, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_points():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for _, job_ms, value in res:
        assert job_ms == 125.0                                # max over ranks, on every rank
        assert value == pytest.approx(2 * 1000 * 50 * 3 / 0.125)


def test_single_rank_needs_no_group():
    assert replicas.max_over_ranks(7.5) == 7.5
    assert replicas.job_throughput(4, 5, 2, 1, 1000.0) == pytest.approx(40.0)
    with pytest.raises(ValueError):
        replicas.job_throughput(4, 5, 2, 1, 0.0)


def test_dist_env_reads_torchrun_variables(monkeypatch):
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert replicas.dist_env() == (3, 4, 1)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k)
    assert replicas.dist_env() == (0, 1, 0)

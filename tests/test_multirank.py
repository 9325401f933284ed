"""The N > 1 host path of bench.py on CPU: replicas (one per GPU, no data-path collective) reduce their
step times with an element-wise maximum over ranks and report whole-job throughput; the reference arm
runs on rank 0 only.  Two gloo ranks on 127.0.0.1 stand in for the torchrun launch."""
import argparse
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r reports times (1 + r, 5 - r, 3): the maxima are (world, 5, 3) on every rank
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 3.0], world)
        q.put((rank, got, bench._env_rank()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (got, env)) for r, got, env in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        got, env = res[r]
        assert got == [2.0, 5.0, 3.0]
        assert env == (r, 2, r)


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]


def test_replica_rate_is_whole_job_throughput():
    # 4 replicas of 1e6 cells each, the slowest taking 1000 ms: 4 M cells/s
    assert bench.replica_rate(1e6, 1000.0, 4) == pytest.approx(4.0)
    assert bench.replica_rate(442368, 0.25, 1) == pytest.approx(1769.472)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""

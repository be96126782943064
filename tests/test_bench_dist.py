"""Host logic of the multi-process bench path, run as world-size-2 gloo
process groups on the CPU: every rank reads its rank from the torchrun
environment, the job time is the slowest rank's, the job value counts all
ranks' units, and the reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.rank_env()
        t = bench.max_over_ranks(1.0 + 0.5 * r, w, device="cpu")   # rank 1 is the slow one
        q.put((r, w, t, bench.job_value(100.0, t, w)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    for r, w, t, v in out:
        assert w == 2 and t == 1.5
        assert v == pytest.approx(2 * 100.0 / 1.5)


def test_job_value_single_rank():
    import bench
    assert bench.job_value(77247 * 50, 0.085, 1) == pytest.approx(77247 * 50 / 0.085)
    assert bench.max_over_ranks(3.0, 1) == 3.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""


def test_learned_flop_count():
    import bench
    fwd, step = bench.learned_flops_per_sample(40, 32)
    # three convolutions: 40x40x64x288, 20x20x64x576, 10x10x64x576 MACs, plus the dense head
    assert fwd == 2 * (40 * 40 * 64 * 288 + 20 * 20 * 64 * 576 + 10 * 10 * 64 * 576 + 6400 * 4)
    assert step > 2 * fwd

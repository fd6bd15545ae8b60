"""Host logic of bench.py's multi-rank path on the CPU (two gloo ranks).

The benchmark runs N independent replicas (one per GPU, no data-path
collective); what needs checking is the process-group setup, the barrier
around the timed region, the max over ranks of the elapsed time, the
whole-job value, and that only rank 0 runs the reference arm.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_init(None)
    bench.barrier(w)
    elapsed = bench.max_over_ranks(10.0 + 5.0 * r, w)      # rank 1 is the slow one
    value = bench.job_value(2_000_000, w, elapsed)
    bench.barrier(w)
    q.put((r, w, dist.get_backend(), elapsed, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_job_value():
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
    for r, (rank, world, backend, elapsed, value) in enumerate(out):
        assert rank == r and world == 2 and backend == "gloo"
        assert elapsed == 15.0                              # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 2_000_000 / 15e-3 / 1e9)


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_init(None) == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(10 ** 9, 1, 1000.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) is None
    assert capsys.readouterr().out == ""

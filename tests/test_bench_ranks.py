"""The multi-rank logic of bench.py (replicas, no data-path collective) on
CPU: world_size 2 over gloo, rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = 100.0 + 50.0 * r  # rank 1 is the slower replica
    worst = bench.max_over_ranks(ms, w, device="cpu")
    rate = bench.job_rate(w, 3 * 1000, worst)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, local, worst, rate))


def test_two_replicas_report_slowest_time_and_job_rate():
    import torch.multiprocessing as mp

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
    for r, (rank, local, worst, rate) in enumerate(out):
        assert rank == r and local == r
        assert worst == 150.0
        assert rate == pytest.approx(2 * 3000 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_rate(1, 1000, 500.0) == pytest.approx(2000.0)


def test_oracle_iteration_time_accepts_zero_iterations():
    """The reference arm's warm-up may be empty (--warmup 0)."""
    import bench
    import oracle
    import synth

    g = synth.grid2d(8, 8)
    aff = oracle.preprocess(g.row_ptr, g.col, 5.0)
    assert bench.oracle_iteration_time(g, aff, 0, 200.0) >= 0.0
    assert bench.oracle_iteration_time(g, aff, 1, 200.0) > 0.0

"""The benchmark's multi-rank path on CPU: gloo, world size 2.

Rays are independent, so N GPUs run N replicas with no data-path collective;
the ranks only agree on the slowest rank's time (a max all-reduce after a
barrier), and the job's throughput counts every rank's rays. The reference
arm runs on rank 0 alone.
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    ms = bench.reduce_max(10.0 + 3.0 * rank, "cpu")
    q.put((r, w, local, ms, bench.job_throughput(w, 2_073_600, 4, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time():
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
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    for o in out:
        assert o[3] == 13.0                                     # the slower rank's time
        assert o[4] == pytest.approx(2 * 2_073_600 * 4 / 13e-3 / 1e6)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(7.5, "cpu") == 7.5
    assert bench.job_throughput(1, 1000, 2, 4.0) == pytest.approx(0.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""

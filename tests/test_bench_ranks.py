"""The bench's N-GPU logic on the host, with two gloo ranks on the CPU: each
rank reconstructs its own noise realisation (replicas: the path has no
exchange step), the job's time is the slowest rank's, and the value counts
the units of all ranks; the reference arm works on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 25.0 * rank
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out.put((rank, t, bench.replica_noise_seed(7, rank), bench.whole_job_value(world, 3, 1200, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
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
    (r0, t0, s0, v0), (r1, t1, s1, v1) = res
    assert t0 == t1 == 125.0
    assert s0 != s1
    assert v0 == pytest.approx(2 * 3 * 1200 / 0.125)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(workload="fan", warmup=1, steps=1, gpus=2)
    assert bench.run_reference(ns) == 0  # returns at once: no scan is generated on rank 1

"""The N > 1 path of bench.py on host cores: two ranks over gloo.

With N GPUs every rank solves its own replica of the workload (no exchange step on the data
path); the ranks meet only at barriers and in the max over ranks of the timings, and rank 0
prints the line. Checked here: both ranks see the slowest rank's time, the whole-job figures
count every replica, and the reference arm leaves ranks other than 0 without work.
"""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    try:
        w, r, local = bench.dist_setup(world, backend="gloo")
        ms = bench.barrier_max(times[r], w)
        q.put((r, w, local, ms, bench.replica_fields(w, ms)))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica_and_count_all_replicas():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [38.2, 41.5]  # rank 1 is the slower replica
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for r, (rank, world, local, ms, fields) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert ms == max(times)
        assert fields == {"n_gpus": 2, "solves_per_s": round(2 * 1e3 / max(times), 3), "parallelism": "replicas x2"}


def test_single_process_needs_no_process_group():
    import bench

    assert bench.barrier_max(12.5, 1) == 12.5
    assert bench.replica_fields(1, 40.0) == {"n_gpus": 1, "solves_per_s": 25.0, "parallelism": "single GPU"}


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    # rank 1 returns before it reads any argument or touches the oracle
    assert bench.run_reference(argparse.Namespace()) is None

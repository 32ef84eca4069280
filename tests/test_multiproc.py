"""The multi-rank path of bench.py on CPU (gloo, world size 2): ranks are
independent replicas; the only exchanges are the barrier and the
max-over-ranks reduction of the timing, and rank 0 alone reports."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.world_info()
        assert (w, r, local) == (world, rank, rank)
        ms = 100.0 + 37.5 * rank                      # the ranks took different times
        dist.barrier()
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.job_rate(30, w, ms_max)
        queue.put((rank, ms_max, value, bench.replica_seed(0, rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_the_slowest_rank_and_rate_counts_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    queue = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(world, _free_port(), queue), nprocs=world, join=True, start_method="spawn")
    out = sorted(queue.get() for _ in range(world))
    assert [o[1] for o in out] == [137.5, 137.5]
    assert all(o[2] == pytest.approx(30 * 2 / 0.1375) for o in out)
    assert out[0][3] != out[1][3]                    # each replica tracks its own sequence


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(gpus=2, steps=1, warmup=0, impl="reference", variant=0, update_mode=0,
                            compose_mode=1, seed=0, no_e2e=True, no_cpu_baseline=True, ref_particles=8)
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""

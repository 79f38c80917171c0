"""The multi-GPU form of bench.py is replicas only: every rank runs the whole
workload, the job's time is the slowest rank's and its work the sum over
ranks.  These tests run that reduction, and the reference arm's rank
handling, as two gloo ranks on the CPU (127.0.0.1)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    assert bench.dist_env() == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 100 (r + 1) units, end to end 2 + r seconds for 10 units
        got = bench.reduce_over_ranks(dist, torch.device("cpu"), 1.0 + rank, 100 * (rank + 1), 2.0 + rank, 10)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (2.0, 300, 3.0, 20)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_oracle_shards_add_up_to_the_whole_sample():
    """The all-threads CPU baseline splits the items into shards of whole
    multiples of the rank count: every item keeps its start rank and its hops
    depend on its own payload only, so the shards' forwarded counts must add
    up to the single-threaded count (ragged last shard included)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_30294_gb300 import inputs

    items = inputs.c1_items(3 * 1024 + 64 * 5, seed=bench.SEED)
    one = bench.oracle_sample_step(items, 1)
    assert one > 0
    for threads in (2, 3, 8):
        assert bench.oracle_sample_step(items, threads) == one


def test_reference_arm_uses_every_host_thread(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "SAMPLE_ITEMS", 4096)

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args()) == 0
    line = json.loads(capsys.readouterr().out)
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == bench.host_threads()
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_repeat_for_runs_until_the_time_is_spent():
    sys.path.insert(0, ROOT)
    import bench

    calls = []
    r, runs, dt = bench.repeat_for(lambda: calls.append(1) or len(calls), min_s=0.05)
    assert runs == len(calls) == r and dt >= 0.05


def test_subset_oracle_legs_on_small_inputs(monkeypatch):
    """The cpu_baseline leg's streamline and transport subsets: the threaded
    shards trace exactly the particles and paths of the single-threaded call."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import oracle
    from paper_2605_30294_gb300 import inputs

    monkeypatch.setattr(bench, "C2_ORACLE_SEEDS", 64)
    monkeypatch.setattr(bench, "C4_ORACLE_CROP", 8)
    field, _ = inputs.c2_field(32)
    seeds = inputs.c2_seeds(640, 32, seed=2)
    r = bench.oracle_c2_subset(field, seeds, 8)
    want = int(oracle.c2_trace(field, seeds[::10][:64], 8)["steps"].astype(np.int64).sum())
    assert r["cores"] == bench.host_threads() and f"{want} particle-steps per run" in r["sample"]
    assert r["particle_steps_per_s"] > 0
    vol, smax = inputs.c4_volume(32)
    view = inputs.c4_views(32, sizes=((16, 16),))[0]
    t = bench.oracle_c4_subset(vol, smax, view, 2)
    assert t["paths_per_s"] > 0 and "(128 paths per run)" in t["sample"]

"""The multi-rank host logic of bench.py on CPU: two gloo ranks (world
size 2).  Each rank gets an independent batch of the same workload, the
timing is reduced to the slowest rank, and the whole-job rate counts the
units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        dev = torch.device("cpu")
        res = {}
        for name in ("c2", "c4"):
            res[name] = [g["seed"] for g in bench.rank_groups(W.config(name, steps_scale=0.001), rank)]
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
        res["max_ms"] = bench.max_over_ranks(ms, dev, world)
        res["rate"] = bench.whole_job_rate(1000.0, world, res["max_ms"])
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    r0, r1 = res
    # the slowest rank's time, seen identically by both ranks
    assert r0["max_ms"] == r1["max_ms"] == 15.0
    assert r0["rate"] == r1["rate"] == pytest.approx(1000.0 * 2 / 15e-3)
    for name in ("c2", "c4"):
        s0, s1 = set(r0[name]), set(r1[name])
        assert len(s0) == len(r0[name]) and len(s1) == len(r1[name])
        assert not (s0 & s1)                          # independent batches


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu"), 1) == 3.5
    assert bench.whole_job_rate(100.0, 1, 10.0) == pytest.approx(1e4)

"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks check the
max-over-ranks timing reduction, the whole-job throughput and that every
rank smooths its own sequence (weak scaling, no data-path collective); the
reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = load_bench()
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slowest
    m = b.max_over_ranks(dist, ms, "cpu")
    y = W.simulate(W.cv_model(), 64, seed=b.rank_sequence_seed(rank))
    got = [None] * world
    dist.all_gather_object(got, float(y[0, 0]))
    out.put((rank, m, b.job_rate(world, 4, 1000, m), got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate, first in res:
        assert m == 15.0                          # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 4 * 1000 / 15e-3)
        assert first[0] != first[1]               # each rank has its own sequence


def test_single_process_reduction():
    b = load_bench()
    assert b.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert b.job_rate(1, 10, 1 << 20, 2.0) == pytest.approx(10 * (1 << 20) / 2e-3)


def test_reference_arm_only_on_rank_zero(capsys):
    import argparse
    b = load_bench()
    args = argparse.Namespace(T=1 << 10, steps=1, warmup=0, precision="fp32", op="rts", scan="auto")
    assert b.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""

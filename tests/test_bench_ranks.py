"""bench.py's multi-rank path on CPU: two gloo ranks reduce their timings and
units the way the GPU job does (slowest rank's time, units summed over
ranks), simulate independent realisations, and only rank 0 runs the
reference arm."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from inputs import C1
from inputs.workloads import c4_ensemble
from inputs.zeldovich import zeldovich_ios


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ranks = bench.Ranks(dist, "cpu")
        ms = [12.5, 20.0][rank]
        units = [1000.0, 1000.0][rank]
        ranks.barrier()
        slow = ranks.max(ms)
        total = ranks.sum(units)
        value = bench.job_throughput(total, slow / 1e3)
        w = bench.replica_workload(C1, rank)
        st = zeldovich_ios(w.with_(n_p=8, n_ios=8))
        share = bench.ensemble_share(c4_ensemble(), world, rank)
        out.put((rank, ranks.world, ranks.rank, slow, total, value, w.seed,
                 st["off"].tobytes(), share))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_gpu_job():
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
    (r0, w0, k0, slow0, tot0, v0, seed0, off0, sh0), (r1, w1, k1, slow1, tot1, v1, seed1, off1, sh1) = res
    assert (w0, w1, k0, k1) == (2, 2, 0, 1)
    # every rank sees the slowest time and the sum of the units
    assert slow0 == slow1 == 20.0 and tot0 == tot1 == 2000.0
    assert v0 == v1 == pytest.approx(2000.0 / 0.020)
    # rank 0 runs the workload itself, rank 1 another realisation of it
    assert seed0 == C1.seed and seed1 != seed0
    assert off0 != off1
    # the ensemble's boxes split over the two ranks: disjoint, complete, balanced
    ws = c4_ensemble()
    assert sorted(sh0 + sh1) == list(range(len(ws))) and not set(sh0) & set(sh1)
    from paper_2512_12629_gb300 import cube2
    cost = [cube2.config_cost(cube2.make_config(w)) for w in ws]
    l0, l1 = sum(cost[i] for i in sh0), sum(cost[i] for i in sh1)
    assert abs(l0 - l1) <= max(cost)


def test_single_rank_reductions_are_identity():
    r = bench.Ranks(None)
    assert (r.world, r.rank) == (1, 0)
    assert r.max(3.5) == 3.5 and r.sum(7.0) == 7.0
    r.barrier()
    assert bench.replica_workload(C1, 0) is C1


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), C1)
    assert capsys.readouterr().out == ""

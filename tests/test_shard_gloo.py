"""Multi-process sharding of one estimate (Section 3.3: only per-observation
averages travel to the master), run as two gloo ranks on the CPU.  Each rank
evaluates its contiguous path range with the oracle; the merged estimate must
equal the single-process estimate over all paths."""
import os
import socket

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from paper_1808_10580_gb300.shard import (allreduce_estimate, estimate_from_partials, merge_estimates, partials,
                                          shard_paths)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, M, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = inputs.plain_fp64_k2()
    off, cnt = shard_paths(M, rank, world)
    g = oracle.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, i0=off, npaths=cnt, nthreads=2)
    mean, var, _ = oracle.estimate(g)
    parts = [None] * world
    dist.all_gather_object(parts, (cnt, mean, var))
    if rank == 0:
        q.put(merge_estimates(parts))
    dist.barrier()
    dist.destroy_process_group()


def _allreduce_worker(rank, world, port, M, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = inputs.plain_fp64_k2()

    def evaluate(off, cnt):
        g = oracle.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, i0=off, npaths=cnt, nthreads=2)
        mean, var, _ = oracle.estimate(g)
        return mean, var

    mean, var = allreduce_estimate(evaluate, M)
    q.put((rank, mean, var))
    dist.barrier()
    dist.destroy_process_group()


def test_partials_round_trip_and_sum_like_pooled_paths():
    rng = np.random.default_rng(4)
    g = rng.normal(0.3, 1.5, size=(5, 77))
    tot = sum(partials(b - a, g[:, a:b].mean(1), g[:, a:b].var(1, ddof=1)) for a, b in ((0, 20), (20, 41), (41, 77)))
    mean, var = estimate_from_partials(tot)
    np.testing.assert_allclose(mean, g.mean(1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(var, g.var(1, ddof=1), rtol=1e-13)


def test_shard_ranges_cover_paths_once():
    for M in (1, 7, 1000, 10_001):
        for world in (1, 2, 3, 8):
            rngs = [shard_paths(M, r, world) for r in range(world)]
            assert rngs[0][0] == 0
            assert all(a[0] + a[1] == b[0] for a, b in zip(rngs, rngs[1:]))
            assert rngs[-1][0] + rngs[-1][1] == M


def test_merge_matches_pooled_statistics():
    rng = np.random.default_rng(3)
    g = rng.normal(1.0, 2.0, size=(4, 101))
    parts = []
    for a, b in ((0, 30), (30, 31), (31, 101)):
        seg = g[:, a:b]
        parts.append((b - a, seg.mean(1), seg.var(1, ddof=1) if b - a > 1 else np.zeros(4)))
    n, m, v = merge_estimates(parts)
    assert n == 101
    assert np.allclose(m, g.mean(1), rtol=1e-14) and np.allclose(v, g.var(1, ddof=1), rtol=1e-13)


def test_two_gloo_ranks_reproduce_single_process_estimate(orc):
    import torch.multiprocessing as mp
    M = 200
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, M, q)) for r in range(2)]
    for p in procs:
        p.start()
    n, mean, var = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = inputs.plain_fp64_k2()
    (rm, rv, _), _ = orc.timedep_estimate(w, npaths=M)
    assert n == M
    assert np.allclose(mean, rm, rtol=0, atol=1e-15) and np.allclose(var, rv, rtol=1e-12)


def test_two_gloo_ranks_allreduce_the_partials(orc):
    # the all-reduce of (n, sum g, sum g^2) over two ranks gives every rank the
    # single-process estimate over all paths
    import torch.multiprocessing as mp
    M = 201
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_allreduce_worker, args=(r, 2, port, M, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = inputs.plain_fp64_k2()
    (rm, rv, _), _ = orc.timedep_estimate(w, npaths=M)
    for _, mean, var in got:
        np.testing.assert_allclose(mean, rm, rtol=0, atol=1e-14)
        np.testing.assert_allclose(var, rv, rtol=1e-12)
    np.testing.assert_array_equal(got[0][1], got[1][1])

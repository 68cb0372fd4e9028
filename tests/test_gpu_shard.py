"""One estimate split over ranks with an all-reduce of the per-observation
partials (Section 3.3), on the GPU path: a one-rank NCCL group through the
library (the glue: path offsets, flags, device partials), and two shards run
one after the other on this GPU whose partials, summed, equal one call over
all paths.  More ranks than GPUs are not emulated on one GPU; the two-rank
exchange itself is tested with gloo ranks in test_shard_gloo.py."""
import os
import socket

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs, shard
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def _arrays(w, obs):
    x = torch.from_numpy(np.ascontiguousarray(w.x[obs])).cuda()
    t = torch.from_numpy(np.ascontiguousarray(w.t[obs])).cuda()
    return x, t, pm.Field(w.K, w.u), pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)


@pytest.mark.parametrize("flags", [pm.PM_FP32 | pm.PM_TENSOR, pm.PM_FP64])
def test_two_shards_sum_to_one_call(c, flags):
    w = inputs.timedep_k10(M=3001) if flags != pm.PM_FP64 else inputs.plain_fp64_k2()
    obs = np.arange(0, len(w.t), max(1, len(w.t) // 30))
    x, t, fld, th = _arrays(w, obs)
    n = len(obs)
    ref_m, ref_v = _gpu.timedep(c, w, flags, obs=obs)
    tot = 0
    for rank in range(2):
        off, cnt = shard.shard_paths(w.M, rank, 2)
        m = torch.empty(n, dtype=torch.float64, device="cuda")
        v = torch.empty_like(m)
        pm.pm_forward_timedep(c, fld, w.kappa, th, x, t, n, cnt, w.dt, w.seed, flags, m, v, path_offset=off)
        tot = tot + shard.partials(cnt, m.cpu().numpy(), v.cpu().numpy())
    mean, var = shard.estimate_from_partials(tot)
    np.testing.assert_allclose(mean, ref_m, rtol=0, atol=1e-13)
    np.testing.assert_allclose(var, ref_v, rtol=1e-10)


def test_one_rank_nccl_group_through_the_library(c):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(_free_port())
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        w = inputs.timedep_k10(M=2000)
        obs = np.arange(0, 300, 10)
        x, t, fld, th = _arrays(w, obs)
        mean, var = shard.timedep_sharded(c, fld, w.kappa, th, x, t, w.M, w.dt, w.seed, pm.PM_FP32 | pm.PM_TENSOR)
        ref_m, ref_v = _gpu.timedep(c, w, pm.PM_FP32 | pm.PM_TENSOR, obs=obs)
        np.testing.assert_allclose(mean, ref_m, rtol=0, atol=1e-14)
        np.testing.assert_allclose(var, ref_v, rtol=1e-12)
    finally:
        dist.destroy_process_group()

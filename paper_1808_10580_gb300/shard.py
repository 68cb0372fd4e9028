"""Host logic for splitting one forward-map estimate over several GPUs.

Section 3.3 of the paper: the particles of an observation are independent and
only the per-observation averages need to reach the master process.  A shard
runs paths [offset, offset + count) of every observation (the RNG is keyed by
the path index, so the union of the shards is exactly the single-GPU run);
the shards' (count, mean, variance) triples are merged in rank order with the
pairwise update of Chan, Golub & LeVeque (1979) (merge_estimates), or summed
over the ranks as per-observation partials {n, sum g, sum g^2} by one
all-reduce (allreduce_estimate: NCCL for device tensors, gloo for host ones).
"""
from __future__ import annotations

import numpy as np


def shard_paths(M: int, rank: int, world: int):
    """Contiguous path range (offset, count) of `rank` out of `world` shards of M paths."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(M, world)
    offset = rank * base + min(rank, extra)
    return offset, base + (1 if rank < extra else 0)


def merge_estimates(parts):
    """Merges [(count, mean[n_obs], var[n_obs]), ...] in order -> (count, mean, var).

    var is the unbiased sample variance (n - 1) of each part and of the result."""
    n_tot = 0
    mean = None
    m2 = None
    for n, mu, var in parts:
        mu = np.asarray(mu, dtype=np.float64)
        var = np.asarray(var, dtype=np.float64)
        if n == 0:
            continue
        m2_b = var * (n - 1)
        if n_tot == 0:
            n_tot, mean, m2 = n, mu.copy(), m2_b.copy()
            continue
        n_new = n_tot + n
        delta = mu - mean
        mean = mean + delta * (n / n_new)
        m2 = m2 + m2_b + delta * delta * (n_tot * n / n_new)
        n_tot = n_new
    if n_tot == 0:
        raise ValueError("no paths")
    var = m2 / (n_tot - 1) if n_tot > 1 else np.zeros_like(m2)
    return n_tot, mean, var


def partials(count, mean, var):
    """Per-observation partial sums [3, n_obs] = (n, sum g, sum g^2) of a shard
    of `count` paths with sample mean `mean` and unbiased variance `var`."""
    mean = np.asarray(mean, dtype=np.float64)
    var = np.asarray(var, dtype=np.float64)
    n = float(count)
    return np.stack([np.full_like(mean, n), n * mean, (n - 1.0) * var + n * mean * mean])


def estimate_from_partials(p):
    """(mean, unbiased variance) from summed partials [3, n_obs].  The variance
    is (sum g^2 - (sum g)^2 / n) / (n - 1) in double precision: its relative
    rounding error grows like 1e-16 (mean / std)^2, negligible for the maps'
    values (|mean| of the order of the standard deviation)."""
    n, s1, s2 = (np.asarray(a, dtype=np.float64) for a in p)
    if np.any(n < 1):
        raise ValueError("no paths")
    mean = s1 / n
    var = np.where(n > 1, (s2 - s1 * mean) / np.maximum(n - 1.0, 1.0), 0.0)
    return mean, var


def allreduce_estimate(evaluate, M, group=None, device=None):
    """One estimate over the ranks of a torch.distributed group (Section 3.3:
    only per-observation sums leave a GPU).  Rank r evaluates paths
    shard_paths(M, r, world) with ``evaluate(offset, count) -> (mean, var)``
    (for the CUDA library: a forward call with path_offset = offset and
    M = count, whose paths are those of one call over all M); the partials
    (n, sum g, sum g^2) of every observation are summed by one all-reduce
    (NCCL when ``device`` is a CUDA device, gloo for the CPU) and every rank
    returns (mean, var) of all M paths."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    offset, count = shard_paths(M, rank, world)
    mean, var = evaluate(offset, count) if count > 0 else (None, None)
    if mean is None:
        raise ValueError("every rank needs at least one path (M >= world size)")
    p = torch.from_numpy(partials(count, mean, var))
    if device is not None:
        p = p.to(device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM, group=group)
    return estimate_from_partials(p.cpu().numpy())


def timedep_sharded(ctx, field, kappa, theta0, x, t, M, dt, seed, flags, group=None, instance=0):
    """Algorithm 1 for one set of observations, its M paths split over the
    ranks of `group` (one GPU per rank, context `ctx` on it): device arrays x,
    t; returns (mean, var) on every rank.  Float, double and tensor-core flags
    as for pm_forward_timedep; PM_DEVICE_PTRS is implied."""
    import torch

    from . import _lib as pm

    n_obs = int(t.shape[0])

    def evaluate(offset, count):
        mean = torch.empty(n_obs, dtype=torch.float64, device=x.device)
        var = torch.empty_like(mean)
        pm.pm_forward_timedep(ctx, field, kappa, theta0, x, t, n_obs, count, dt, seed,
                              (flags | pm.PM_DEVICE_PTRS) & ~pm.PM_ASYNC, mean, var, path_offset=offset,
                              instance=instance)
        return mean.cpu().numpy(), var.cpu().numpy()

    return allreduce_estimate(evaluate, M, group=group, device=x.device)

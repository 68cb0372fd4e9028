"""Host logic for splitting one forward-map estimate over several GPUs.

Section 3.3 of the paper: the particles of an observation are independent and
only the per-observation averages need to reach the master process.  A shard
runs paths [offset, offset + count) of every observation (the RNG is keyed by
the path index, so the union of the shards is exactly the single-GPU run);
the shards' (count, mean, variance) triples are merged in rank order with the
pairwise update of Chan, Golub & LeVeque (1979).
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

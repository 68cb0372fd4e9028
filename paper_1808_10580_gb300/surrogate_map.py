"""Gradient-based MAP estimation on the learned surrogate of the forward map.

The particle estimator of G(u) is a Monte Carlo average with no Frechet
derivative in u (the limitation Section 3 of the paper notes for the particle
method), so derivative-based optimisation of the posterior cannot run on it
directly.  The surrogate network is differentiable: with the Gaussian prior
N(0, diag(s^2)) of the pCN sampler and data y with noise sigma, the MAP point
of the surrogate posterior minimises

    J(u) = sum_j (y_j - Y_j(z))^2 / (2 sigma^2) + (1/2) sum_k (u_k / s_k)^2,
    z = (u - shift) * scale   (the network's input coordinates),

whose gradient is dJ/du = -scale * J_z(z)^T (y - Y(z)) / sigma^2 + u / s^2,
the first term one vector-Jacobian product of the network
(pm_surrogate_input_gradient).  The iteration runs in whitened coordinates
w = u / s (the prior term becomes |w|^2 / 2) with Adam (Kingma & Ba 2015)
steps, for B starting points at once: every iteration is one batched forward
and one batched vector-Jacobian product on the tensor cores.  The particle map
stays the judge: the result is a candidate to evaluate with it (or to start
chains from), not an estimate of G.
"""
from __future__ import annotations

import numpy as np

from . import _lib as pm


def objective(ctx, net, u, y, sigma, prior_std, shift=None, scale=None):
    """J(u) for every row of u [B, n_u] through the surrogate -> [B]."""
    u = np.asarray(u, dtype=np.float64)
    z = _inputs(u, shift, scale)
    Y = np.empty((u.shape[0], len(y)), np.float32)
    pm.pm_surrogate_infer(ctx, net, z, Y)
    r = np.asarray(y)[None, :] - Y.astype(np.float64)
    return 0.5 * (r ** 2).sum(1) / sigma ** 2 + 0.5 * ((u / prior_std) ** 2).sum(1)


def gradient(ctx, net, u, y, sigma, prior_std, shift=None, scale=None):
    """(J(u), dJ/du) for every row of u [B, n_u]."""
    u = np.asarray(u, dtype=np.float64)
    B = u.shape[0]
    z = _inputs(u, shift, scale)
    Y = np.empty((B, len(y)), np.float32)
    pm.pm_surrogate_infer(ctx, net, z, Y)
    r = np.asarray(y)[None, :] - Y.astype(np.float64)
    dY = (-r / sigma ** 2).astype(np.float32)
    dz = np.empty(z.shape, np.float32)
    pm.pm_surrogate_input_gradient(ctx, net, z, dY, dz)
    sc = 1.0 if scale is None else np.asarray(scale, dtype=np.float64)[None, :]
    J = 0.5 * (r ** 2).sum(1) / sigma ** 2 + 0.5 * ((u / prior_std) ** 2).sum(1)
    return J, dz.astype(np.float64) * sc + u / prior_std ** 2


def map_estimate(ctx, net, y, sigma, prior_std, u0, shift=None, scale=None, steps=300, lr=0.05, lr_decay=0.99,
                 beta1=0.9, beta2=0.999, eps=1e-8):
    """Minimises J from every row of u0 [B, n_u] by `steps` Adam steps in w = u / s
    (step size lr lr_decay^k) -> (u [B, n_u], J(u) [B])."""
    s = np.asarray(prior_std, dtype=np.float64)
    w = np.asarray(u0, dtype=np.float64) / s
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    a = lr
    for k in range(1, steps + 1):
        _, g = gradient(ctx, net, w * s, y, sigma, s, shift, scale)
        gw = g * s  # dJ/dw
        m = beta1 * m + (1 - beta1) * gw
        v = beta2 * v + (1 - beta2) * gw * gw
        w = w - a * (m / (1 - beta1 ** k)) / (np.sqrt(v / (1 - beta2 ** k)) + eps)
        a *= lr_decay
    u = w * s
    return u, objective(ctx, net, u, y, sigma, s, shift, scale)


def _inputs(u, shift, scale):
    z = u if shift is None else u - np.asarray(shift, dtype=np.float64)[None, :]
    if scale is not None:
        z = z * np.asarray(scale, dtype=np.float64)[None, :]
    return np.ascontiguousarray(z, dtype=np.float32)

"""Surrogate-screened pCN over the particle forward map (the paper's use of the
map inside MCMC, Section 4.1, with a learned pre-screen).

Workflow, all on the GPU through the library's C ABI:
  1. the forward map G: the time-dependent map of the 256-instance batched
     workload's first instance (10 x 10 grid, t_j in {0.25, 0.5, 0.75, 1} by
     (i + j) mod 4, kappa = 0.01, dt = 1e-3, M = 4096 particles per observation),
     every evaluation on one RNG stream and seed, so G is a deterministic
     function of u (common random numbers);
  2. data y = G(u_true) + N(0, sigma^2 I), u_true a prior draw;
  3. training pairs (u, G(u)) with u from the prior, or local to the chains'
     start state, evaluated 256 at a time by the batched map;
  4. the surrogate network trained on (standardised u, G(u)): u / prior std,
     or (u - start) / (spread * prior std) for local pairs;
  5. pCN chains, plain and with delayed acceptance through the surrogate, with
     the same beta, compared by accepted proposals per second.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import _lib as pm
from . import inputs


@dataclass
class Problem:
    K: int
    x: np.ndarray
    t: np.ndarray
    theta0: inputs.Fourier
    kappa: float
    dt: float
    M: int
    path_seed: int
    std: np.ndarray          # prior standard deviation per coefficient
    y: np.ndarray = None
    u_true: np.ndarray = None
    sigma: float = 0.01


def prior_std(K: int) -> np.ndarray:
    k = inputs.half_mode_list(K).astype(np.float64)
    return np.repeat(((k ** 2).sum(1)) ** -1.0, 2)


def make_problem(M: int = 4096, sigma: float = 0.01, seed_true: int = 5004, seed_noise: int = 6004) -> Problem:
    w = inputs.batched_instances(B=1, M=M)[0]
    return Problem(K=w.K, x=w.x, t=w.t, theta0=w.theta0, kappa=w.kappa, dt=w.dt, M=w.M, path_seed=w.seed,
                   std=prior_std(w.K), sigma=sigma)


def forward_many(ctx, prob: Problem, U: np.ndarray, chunk: int = 256, tensor: bool = True) -> np.ndarray:
    """G(u) for every row of U [N, n_u] with the batched map (one stream, one seed);
    the velocity sum on the tensor cores unless tensor=False."""
    n_obs = len(prob.t)
    out = np.empty((U.shape[0], n_obs))
    th = pm.Fourier(prob.theta0.k, prob.theta0.a, prob.theta0.b)
    for s in range(0, U.shape[0], chunk):
        part = U[s:s + chunk]
        B = part.shape[0]
        inst = [dict(kind=pm.PM_KIND_TIMEDEP, u=part[b], kappa=prob.kappa, dt=prob.dt, row0=b * n_obs, n_obs=n_obs,
                     M=prob.M, seed=prob.path_seed, stream=0) for b in range(B)]
        x = np.ascontiguousarray(np.tile(prob.x, (B, 1)))
        t = np.ascontiguousarray(np.tile(prob.t, B))
        batch = pm.Batch(prob.K, inst, x, t, th, None)
        mean = np.empty(B * n_obs)
        pm.pm_forward_batched(ctx, batch, pm.PM_FP32 | (pm.PM_TENSOR if tensor else 0), mean)
        out[s:s + B] = mean.reshape(B, n_obs)
    return out


def make_data(ctx, prob: Problem, seed_true: int = 5004, seed_noise: int = 6004):
    rng = np.random.Generator(np.random.PCG64(seed_true))
    prob.u_true = prob.std * rng.standard_normal(len(prob.std))
    G = forward_many(ctx, prob, prob.u_true[None, :])[0]
    noise = np.random.Generator(np.random.PCG64(seed_noise)).standard_normal(len(G))
    prob.y = G + prob.sigma * noise
    return prob


def training_pairs(ctx, prob: Problem, n: int, seed: int = 7004, center: np.ndarray = None, spread: float = 1.0,
                   tensor: bool = True, coords=None):
    """n pairs (network input, G(u)) with u = center + spread * std * z,
    z ~ N(0, I) (center None: 0, so spread 1 gives prior draws).  The network
    input is (u - shift) * scale for coords = (shift, scale); the default is
    the prior coordinates u / std."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Z = rng.standard_normal((n, len(prob.std)))
    c = np.zeros(len(prob.std)) if center is None else np.asarray(center, dtype=np.float64)
    U = c[None, :] + spread * prob.std[None, :] * Z
    G = forward_many(ctx, prob, U, tensor=tensor)
    shift, scale = coords if coords is not None else screen_coords(prob)
    X = (U - shift[None, :]) * scale.astype(np.float64)[None, :]
    return X.astype(np.float32), G.astype(np.float32)


def screen_coords(prob: Problem, center: np.ndarray = None, spread: float = 1.0):
    """(shift, scale) of the network input (u - shift) * scale: by default the
    prior coordinates u / std; with a center, (u - center) / (spread * std)."""
    shift = np.zeros(len(prob.std)) if center is None else np.asarray(center, dtype=np.float64)
    return shift, (1.0 / (spread * prob.std)).astype(np.float32)


def train_surrogate(ctx, prob: Problem, Z, G, hidden=512, epochs=20, batch=512, lr=1e-3, seed=8004,
                    weight_decay=0.0, lr_decay=1.0):
    net = pm.pm_surrogate_create(ctx, Z.shape[1], hidden, G.shape[1], seed)
    hist = pm.pm_surrogate_train(ctx, net, Z, G, epochs=epochs, batch=batch, lr=lr, shuffle_seed=seed,
                                 weight_decay=weight_decay, lr_decay=lr_decay)
    return net, hist


def surrogate_rmse(ctx, net, Z, G):
    Y = np.empty_like(G)
    pm.pm_surrogate_infer(ctx, net, Z, Y)
    return float(np.sqrt(((Y - G) ** 2).mean()))


def start_states(prob: Problem, n_chains: int, spread: float = 0.0, seed: int = 9004):
    rng = np.random.Generator(np.random.PCG64(seed))
    return prob.u_true[None, :] + spread * prob.std[None, :] * rng.standard_normal((n_chains, len(prob.std)))


def run_chains(ctx, prob: Problem, u0, beta, n_steps, seed, net=None, tensor: bool = True, coords=None):
    """coords: (shift, scale) of the network input (default: prior coordinates u / std)."""
    th = pm.Fourier(prob.theta0.k, prob.theta0.a, prob.theta0.b)
    shift, scale = coords if coords is not None else screen_coords(prob)
    ch = pm.PCN(ctx, prob.K, u0, prob.y, prob.sigma, beta, seed, theta0=th, x=prob.x, t=prob.t, kappa=prob.kappa,
                dt=prob.dt, M=prob.M, path_seed=prob.path_seed, screen=net,
                screen_scale=scale if net is not None else None,
                screen_shift=shift if net is not None else None, tensor=tensor)
    t0 = time.perf_counter()
    st = ch.run(n_steps)
    st["wall_seconds"] = time.perf_counter() - t0
    u, phi, s, n = ch.state()
    ch.close()
    st["mean_phi"] = float(np.mean(phi))
    st["accepted_per_s"] = st["accepts"] / st["wall_seconds"]
    st["sq_jump_per_s"] = st["sq_jump"] / st["wall_seconds"]
    st["samples_per_s"] = st["proposals"] / st["wall_seconds"]
    return st, s / max(n, 1)


def run_chains_tracked(ctx, prob: Problem, u0, beta, n_steps, seed, net=None, tensor: bool = True, coords=None):
    """run_chains, one step at a time, keeping every chain's running sum of
    states: -> (stats, per-chain means [n_chains, n_u])."""
    th = pm.Fourier(prob.theta0.k, prob.theta0.a, prob.theta0.b)
    shift, scale = coords if coords is not None else screen_coords(prob)
    ch = pm.PCN(ctx, prob.K, u0, prob.y, prob.sigma, beta, seed, theta0=th, x=prob.x, t=prob.t, kappa=prob.kappa,
                dt=prob.dt, M=prob.M, path_seed=prob.path_seed, screen=net,
                screen_scale=scale if net is not None else None,
                screen_shift=shift if net is not None else None, tensor=tensor)
    sums = np.zeros_like(np.asarray(u0, dtype=np.float64))
    tot = None
    wall = 0.0
    for _ in range(n_steps):
        t0 = time.perf_counter()
        st = ch.run(1)
        wall += time.perf_counter() - t0
        u, _, _, _ = ch.state()
        sums += u
        if tot is None:
            tot = dict(st)
        else:
            for k in ("steps", "proposals", "stage1_accepts", "accepts", "forward_evals", "seconds", "sq_jump"):
                tot[k] += st[k]
    ch.close()
    tot["wall_seconds"] = wall
    tot["accepted_per_s"] = tot["accepts"] / wall
    tot["samples_per_s"] = tot["proposals"] / wall
    return tot, sums / max(n_steps, 1)


def posterior_mean_error(chain_means):
    """Relative Monte Carlo error of the pooled posterior-mean estimate from
    independent chains: || SE || / || mean || with SE_k the between-chain
    standard deviation of coordinate k over sqrt(chains)."""
    m = np.asarray(chain_means, dtype=np.float64)
    mean = m.mean(0)
    se = m.std(0, ddof=1) / np.sqrt(m.shape[0])
    return float(np.linalg.norm(se) / max(np.linalg.norm(mean), 1e-300)), mean


def misfit(prob: Problem, G):
    """Phi = sum_j (y_j - G_j)^2 / (2 sigma^2) for rows of G [N, n_obs]."""
    return ((prob.y[None, :] - G) ** 2).sum(1) / (2 * prob.sigma ** 2)


def pcn_proposals(prob: Problem, u, beta, n, seed):
    """n pCN proposals sqrt(1 - beta^2) u + beta C^{1/2} xi around u."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sqrt(1 - beta ** 2) * u[None, :] + beta * prob.std[None, :] * rng.standard_normal((n, len(u)))

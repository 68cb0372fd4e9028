"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path's tests/benchmark and by the CPU oracle's
tests.  It draws random parameters and observation layouts only; it contains
none of the method's arithmetic (no velocity, no particle step, no estimator).

Every draw uses numpy's PCG64 generator with a fixed seed, so a workload is a
pure function of its name.  Shapes follow Section 4 of the paper: about 100
observations (Example 1), a Fourier stream function over a square lattice of
wave numbers (Eq. v_expand) with a |k|^-4 prior on each real coefficient,
Dirichlet data on a disk.  The concrete recipe of each workload is in its
function's docstring below.

Layout conventions (the library's input format, shared by both sides):
  * ``u``: float64 array of length 2H, pairs (a_h, b_h) over the half-plane
    lattice {m > 0, |n| <= K} U {m = 0, 0 < n <= K}, ordered by m then n;
  * ``x``: float64 [n_obs, 2]; ``t``: float64 [n_obs];
  * theta0: integer wave vectors [nq, 2] with cosine/sine amplitudes.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


def half_mode_list(K: int) -> np.ndarray:
    """Wave vectors of the coefficient layout, [H, 2] int32, in storage order."""
    out = [(0, n) for n in range(1, K + 1)]
    out += [(m, n) for m in range(1, K + 1) for n in range(-K, K + 1)]
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


def prior_field(K: int, seed: int, scale: float = 1.0, counter: int = 0) -> np.ndarray:
    """Coefficients u with each real a_h, b_h ~ N(0, |k_h|_2^-4), times ``scale``.

    ``counter`` selects an independent draw for the same seed (instance b of a
    batch)."""
    k = half_mode_list(K).astype(np.float64)
    knorm2 = (k ** 2).sum(axis=1)
    rng = np.random.Generator(np.random.PCG64([seed, counter]))
    z = rng.standard_normal((k.shape[0], 2))
    std = knorm2 ** -1.0  # |k|^-2 standard deviation
    return (scale * z * std[:, None]).reshape(-1).astype(np.float64)


def grid_points(n: int) -> np.ndarray:
    """Cell-centred n x n grid on the unit square, row-major, [n*n, 2]."""
    c = (np.arange(n) + 0.5) / n
    xx, yy = np.meshgrid(c, c, indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1).astype(np.float64)


def disk_points(n: int, rmax: float, seed: int) -> np.ndarray:
    """n points uniform in area on the disk r <= rmax."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u1 = rng.random(n)
    u2 = rng.random(n)
    r = rmax * np.sqrt(u1)
    phi = 2.0 * np.pi * u2
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


def random_theta0(nq: int, kmax: int, seed: int):
    """nq distinct half-plane wave vectors with |k|_inf <= kmax, amplitudes
    N(0, 1/nq) each (so that theta0 has unit variance)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cand = half_mode_list(kmax)
    idx = rng.choice(cand.shape[0], size=nq, replace=False)
    k = cand[np.sort(idx)].astype(np.int32)
    a = rng.standard_normal(nq) / np.sqrt(nq)
    b = rng.standard_normal(nq) / np.sqrt(nq)
    return k, a.astype(np.float64), b.astype(np.float64)


@dataclass
class Fourier:
    """theta0(x) = sum_q a_q cos(2 pi k_q.x) + b_q sin(2 pi k_q.x)."""
    k: np.ndarray  # [nq, 2] int32
    a: np.ndarray  # [nq]
    b: np.ndarray  # [nq]


@dataclass
class DirichletData:
    """Disk of radius R; g = quad (y1^2 - y2^2) + sum_m a_m cos(m phi) + b_m sin(m phi); f = f_const."""
    R: float = 1.0
    quad: float = 0.0
    f_const: float = 0.0
    a: np.ndarray = field(default_factory=lambda: np.zeros(0))
    b: np.ndarray = field(default_factory=lambda: np.zeros(0))


@dataclass
class DiffusionForcing:
    """Diagonal affine diffusion sigma_i(x) = s0[i] + s1[i] x_i (with the
    Milstein term when `milstein`) and Gaussian sources F[q] exp(-w |x - c_q|^2)
    added to the constant forcing of the boundary data."""
    s0: np.ndarray
    s1: np.ndarray
    milstein: bool = True
    c: np.ndarray = field(default_factory=lambda: np.zeros((0, 2)))
    F: np.ndarray = field(default_factory=lambda: np.zeros(0))
    w: float = 0.0


@dataclass
class TimedepWorkload:
    name: str
    K: int
    u: np.ndarray
    kappa: float
    theta0: Fourier
    x: np.ndarray
    t: np.ndarray
    M: int
    dt: float
    seed: int


@dataclass
class DirichletWorkload:
    name: str
    K: int
    u: np.ndarray
    drift_scale: float
    kappa: float
    g: DirichletData
    x: np.ndarray
    M: int
    dt: float
    max_steps: int
    seed: int


@dataclass
class SquareBVP:
    """The optimal-forcing boundary-value problem in the unit square (the
    example of Section 4, Eq. bvp:ex1): constant drift b, diffusion kappa,
    Gaussian source profiles exp(-w |x - c_q|^2) at c [n_src, 2], boundary
    data g_cos (cos(pi x1 / 2) + cos(pi x2 / 2)) / 2 + g_quad (x1^2 - x2^2)."""
    b: np.ndarray
    kappa: float
    c: np.ndarray
    w: float
    g_cos: float = 1.0
    g_quad: float = 0.0


@dataclass
class SquareBVPWorkload:
    name: str
    prob: SquareBVP
    x: np.ndarray          # [n_obs, 2] observation points
    y: np.ndarray          # [n_obs] target data
    M: int
    dt: float
    max_steps: int
    seed: int


def optimal_forcing(M: int = 1_000_000) -> SquareBVPWorkload:
    """The paper's optimal-forcing example: b = (1, 1), kappa = 0.282, three
    sources exp(-4 |x - c_q|^2), the paper's boundary data, data y = (0, 0, 0)
    at three observation points.  The paper shows its source and observation
    locations only in a figure; these stand in for them (sources near three
    corners of the square's interior, observations between them).  dt = 1e-4,
    M paths per observation, path seed 4005."""
    prob = SquareBVP(b=np.array([1.0, 1.0]), kappa=0.282,
                     c=np.array([[0.25, 0.25], [0.75, 0.35], [0.4, 0.8]]), w=4.0)
    x = np.array([[0.3, 0.55], [0.65, 0.6], [0.55, 0.25]])
    return SquareBVPWorkload("optimal_forcing_square_3src_3obs", prob, x, np.zeros(3), M, 1e-4, 10_000_000, 4005)


def plain_fp64_k2() -> TimedepWorkload:
    """K=2 (24 reals), kappa=0.05, theta0 = sin 2pi x1 sin 2pi x2, 3x3 grid, t=1, M=1000, dt=0.01."""
    th = Fourier(k=np.array([[1, -1], [1, 1]], dtype=np.int32),
                 a=np.array([0.5, -0.5]), b=np.zeros(2))
    x = grid_points(3)
    return TimedepWorkload("timedep_k2_3x3_t1_M1000_fp64", 2, prior_field(2, 1000), 0.05, th,
                           x, np.ones(len(x)), 1000, 0.01, 4000)


def timedep_k10(M: int = 10_000) -> TimedepWorkload:
    """K=10 (440 reals), kappa=0.01, 16-mode theta0, 10x10 grid x t in {0.25, 0.5, 1},
    M=1e4, dt=1e-3.  Observation index = t_index * 100 + grid index."""
    k, a, b = random_theta0(16, 4, 2001)
    g = grid_points(10)
    times = [0.25, 0.5, 1.0]
    x = np.concatenate([g for _ in times], axis=0)
    t = np.concatenate([np.full(len(g), tt) for tt in times])
    return TimedepWorkload("timedep_k10_300obs_M1e4_dt1e-3", 10, prior_field(10, 1001), 0.01,
                           Fourier(k, a, b), x, t, M, 1e-3, 4001)


def two_point_time_series(K: int = 16, M: int = 100_000) -> TimedepWorkload:
    """The observation layout of the paper's turbulent-flow example (Section
    4, Example 3): 2 locations x 13 times evenly spaced in [0, 0.5] (26
    observations), kappa = 3e-5.  The example's field (|k|_2 <= 80) and data
    are not available; a prior field with |k|_inf <= K (seed 1006) and the
    16-mode theta0 of the 440-mode workload stand in.  dt = 1e-3, path seed 4006."""
    k, a, b = random_theta0(16, 4, 2001)
    pts = np.array([[0.3, 0.6], [0.7, 0.25]])
    times = np.linspace(0.0, 0.5, 13)
    x = np.repeat(pts, len(times), axis=0)
    t = np.tile(times, len(pts))
    return TimedepWorkload(f"two_points_13_times_k{K}_M{M}", K, prior_field(K, 1006), 3e-5, Fourier(k, a, b), x, t, M,
                           1e-3, 4006)


def dirichlet_disk_k10(M: int = 100_000) -> DirichletWorkload:
    """Unit disk, K=10 field x 0.5, kappa=0.05, g = y1^2 - y2^2 + 0.1 sin 3phi,
    50 uniform-area points r <= 0.9, M=1e5, dt=1e-4."""
    g = DirichletData(R=1.0, quad=1.0, f_const=0.0, a=np.zeros(3), b=np.array([0.0, 0.0, 0.1]))
    return DirichletWorkload("dirichlet_disk_k10_50obs_M1e5_dt1e-4", 10, prior_field(10, 1002), 0.5,
                             0.05, g, disk_points(50, 0.9, 3002), M, 1e-4, 10_000_000, 4002)


def dirichlet_general_disk(M: int = 10_000) -> tuple:
    """The disk workload (K=10 field x 0.5, 50 uniform-area points r <= 0.9,
    g = y1^2 - y2^2 + 0.1 sin 3phi, dt = 1e-4) with a state-dependent diffusion
    sigma(x) = diag(0.3 + 0.15 x1, 0.3 - 0.1 x2) (between 0.15 and 0.45 on the
    disk) and three Gaussian sources exp(-4 |x - c|^2) of amplitudes 1, -0.5,
    0.8 at (0.3, 0.2), (-0.4, 0.1), (0, -0.5); Milstein steps.  Returns
    (DirichletWorkload, DiffusionForcing); the workload's kappa is unused."""
    w = dirichlet_disk_k10(M=M)
    w.name = f"dirichlet_general_disk_k10_50obs_M{M}_dt1e-4"
    df = DiffusionForcing(s0=np.array([0.3, 0.3]), s1=np.array([0.15, -0.1]), milstein=True,
                          c=np.array([[0.3, 0.2], [-0.4, 0.1], [0.0, -0.5]]), F=np.array([1.0, -0.5, 0.8]), w=4.0)
    return w, df


def batched_instances(B: int = 256, M: int = 4096, seed: int = 1003):
    """Instance b: even b time-dependent (K=10 field, kappa=0.01, dt=1e-3, 10x10 grid,
    t_j in {0.25, 0.5, 0.75, 1.0} by (i+j) mod 4); odd b Dirichlet (unit disk,
    field x 0.5, kappa=0.05, dt=1e-3, 100 uniform-area points r <= 0.9).
    Each instance draws its own u from the prior (counter b)."""
    k, a, bq = random_theta0(16, 4, 2003)
    theta0 = Fourier(k, a, bq)
    g = DirichletData(R=1.0, quad=1.0, f_const=0.0, a=np.zeros(3), b=np.array([0.0, 0.0, 0.1]))
    grid = grid_points(10)
    tvals = np.array([0.25, 0.5, 0.75, 1.0])
    ij = np.array([(i + j) % 4 for i in range(10) for j in range(10)])
    out = []
    for b in range(B):
        u = prior_field(10, seed, counter=b)
        if b % 2 == 0:
            out.append(TimedepWorkload(f"batched_td_{b}", 10, u, 0.01, theta0, grid.copy(),
                                       tvals[ij].copy(), M, 1e-3, 4003))
        else:
            out.append(DirichletWorkload(f"batched_dir_{b}", 10, u, 0.5, 0.05, g,
                                         disk_points(100, 0.9, 3003 + b), M, 1e-3, 1_000_000, 4003))
    return out

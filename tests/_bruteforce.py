"""Independent float64 numpy restatement of the particle paths, for brute-force
checks of the oracle on tiny inputs (a few paths, a few steps).  Written
separately from oracle/pm_oracle.c: Philox4x32-10 from Salmon et al. (SC'11),
the Box-Muller transform, the stream-function velocity and Euler-Maruyama."""
import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox(ctr, key):
    c = [int(v) & MASK for v in ctr]
    k = [int(v) & MASK for v in key]
    for r in range(10):
        if r:
            k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & MASK, p1 & MASK, ((p0 >> 32) ^ c[3] ^ k[1]) & MASK, p0 & MASK]
    return c


def normals(seed, b, j, i, n):
    r = philox([n // 2, i, j, b], [seed & MASK, seed >> 32])
    ra, rb = (r[0], r[1]) if n % 2 == 0 else (r[2], r[3])
    ua = ((ra >> 9) * 2 + 1) / 2.0 ** 24
    ub = ((rb >> 9) * 2 + 1) / 2.0 ** 24
    rho = math.sqrt(-2.0 * math.log(ua))
    return rho * math.cos(2 * math.pi * ub), rho * math.sin(2 * math.pi * ub)


def modes(K):
    return [(0, n) for n in range(1, K + 1)] + [(m, n) for m in range(1, K + 1) for n in range(-K, K + 1)]


def velocity(K, u, x):
    v1 = v2 = 0.0
    for h, (m, n) in enumerate(modes(K)):
        a, b = u[2 * h], u[2 * h + 1]
        th = 2 * math.pi * (m * x[0] + n * x[1])
        # psi_h = a cos th + b sin th; v = (-d2 psi, d1 psi)
        d = 2 * math.pi * (-a * math.sin(th) + b * math.cos(th))
        v1 += -n * d
        v2 += m * d
    return v1, v2


def timedep_path(K, u, kappa, x0, t, dt, seed, j, i, b=0):
    N = 0 if t <= 0 else math.ceil(t / dt - 1e-9)
    X = [x0[0], x0[1]]
    for n in range(N):
        h = t - (N - 1) * dt if n == N - 1 else dt
        v = velocity(K, u, X)
        xi = normals(seed, b, j, i, n)
        s = math.sqrt(2 * kappa * h)
        X = [X[0] - v[0] * h + s * xi[0], X[1] - v[1] * h + s * xi[1]]
        X = [X[0] - math.floor(X[0]), X[1] - math.floor(X[1])]
    return X


def dirichlet_path(K, u, drift, kappa, R, x0, dt, max_steps, seed, j, i, b=0):
    X = [x0[0], x0[1]]
    n = 0
    s = math.sqrt(2 * kappa * dt)
    while X[0] ** 2 + X[1] ** 2 < R * R and n < max_steps:
        v = velocity(K, u, X)
        xi = normals(seed, b, j, i, n)
        X = [X[0] - drift * v[0] * dt + s * xi[0], X[1] - drift * v[1] * dt + s * xi[1]]
        n += 1
    exited = X[0] ** 2 + X[1] ** 2 >= R * R
    return X, (n if exited else -1)

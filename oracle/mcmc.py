"""Oracle of the pCN sampler and its delayed-acceptance form (TEST INFRASTRUCTURE ONLY).

The paper samples its posteriors with preconditioned Crank-Nicolson MCMC
(Section 4.1) and defers the details; the standard algorithm is restated here:
  * prior N(0, C) with C diagonal, C^{1/2} = diag(std);
  * proposal u' = sqrt(1 - beta^2) u + beta C^{1/2} xi, xi ~ N(0, I);
  * Phi(u) = sum_j (y_j - G_j(u))^2 / (2 sigma^2);
  * plain pCN accepts with probability min(1, exp(Phi(u) - Phi(u'))).
Delayed acceptance (Christen & Fox 2005) screens with a cheap Phi~ first:
  stage 1 accepts with min(1, exp(Phi~(u) - Phi~(u'))); only then is the
  expensive Phi(u') computed and stage 2 accepts with
  min(1, exp(Phi(u) - Phi(u') - Phi~(u) + Phi~(u'))).
Randomness (a reading: the paper fixes none) comes from Philox4x32-10 with the
counter layouts below, so that another implementation can draw the same numbers:
  proposal normals of chain c at step s: counter {s, c, q, 0x4D43}, q = 0, 1, ...;
  the words (r0, r1) and (r2, r3) of each counter give two Box-Muller pairs, i.e.
  normals 4q .. 4q+3;
  stage-1 / stage-2 uniforms: counter {s, c, 0xFFFFFFFF, 1 or 2}, word r0;
  u = (2 (r >> 9) + 1) / 2^24 (never 0 or 1).
"""
import math

import numpy as np

import oracle

TAG_PROPOSAL = 0x4D43
Q_UNIFORM = 0xFFFFFFFF


def prior_std(K):
    """|k_h|^-2 for each real coefficient, in the layout of the field (a_h, b_h pairs)."""
    k = oracle.half_modes(K).astype(np.float64)
    s = ((k ** 2).sum(1)) ** -1.0
    return np.repeat(s, 2)


def _uniform(r):
    return (2.0 * float(int(r) >> 9) + 1.0) / 16777216.0


def proposal_normals(seed, step, chain, n):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    nq = (n + 3) // 4
    ctr = np.array([[step, chain, q, TAG_PROPOSAL] for q in range(nq)], dtype=np.uint32)
    words = oracle.philox(ctr, key)
    out = []
    for w in words:
        for a, b in ((w[0], w[1]), (w[2], w[3])):
            ua, ub = _uniform(a), _uniform(b)
            rho = math.sqrt(-2.0 * math.log(ua))
            out += [rho * math.cos(2 * math.pi * ub), rho * math.sin(2 * math.pi * ub)]
    return np.array(out[:n])


def accept_uniform(seed, step, chain, stage):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w = oracle.philox(np.array([[step, chain, Q_UNIFORM, stage]], dtype=np.uint32), key)[0]
    return _uniform(w[0])


def phi(y, G, sigma):
    r = np.asarray(y, dtype=np.float64) - np.asarray(G, dtype=np.float64)
    return float((r * r).sum() / (2.0 * sigma * sigma))


def run(u0, G, y, sigma, beta, std, n_steps, seed, Gs=None, step0=0):
    """Chains u0 [C, n] for n_steps pCN steps (delayed acceptance when the cheap
    map Gs is given).  Returns the final states, the running sum of states over
    all steps (for posterior means) and counters; sq_jump sums the squared
    prior-whitened jumps |(u' - u) / std|^2 of accepted moves (the expected
    squared jump distance, a standard efficiency measure of a sampler)."""
    U = np.array(u0, dtype=np.float64, copy=True)
    C, n = U.shape
    rho = math.sqrt(1.0 - beta * beta)
    Phi = np.array([phi(y, G(U[c]), sigma) for c in range(C)])
    PhiS = np.array([phi(y, Gs(U[c]), sigma) for c in range(C)]) if Gs else np.zeros(C)
    total = np.zeros(n)
    stats = dict(stage1=0, accepts=0, evals=0, sq_jump=0.0)
    for s in range(step0, step0 + n_steps):
        for c in range(C):
            up = rho * U[c] + beta * std * proposal_normals(seed, s, c, n)
            if Gs is not None:
                phs = phi(y, Gs(up), sigma)
                if accept_uniform(seed, s, c, 1) >= min(1.0, math.exp(min(0.0, PhiS[c] - phs))):
                    continue
                stats["stage1"] += 1
                ph = phi(y, G(up), sigma)
                stats["evals"] += 1
                a = PhiS[c] - phs  # log of the stage-1 ratio
                if accept_uniform(seed, s, c, 2) < math.exp(min(0.0, (Phi[c] - ph) - a)):
                    stats["sq_jump"] += float((((up - U[c]) / std) ** 2).sum())
                    U[c], Phi[c], PhiS[c] = up, ph, phs
                    stats["accepts"] += 1
            else:
                ph = phi(y, G(up), sigma)
                stats["evals"] += 1
                if accept_uniform(seed, s, c, 2) < math.exp(min(0.0, Phi[c] - ph)):
                    stats["sq_jump"] += float((((up - U[c]) / std) ** 2).sum())
                    U[c], Phi[c] = up, ph
                    stats["accepts"] += 1
        total += U.sum(0)
    return U, total, stats


def linear_gaussian_posterior(A, y, sigma, std):
    """Posterior mean and covariance of u ~ N(0, diag(std^2)), y = A u + N(0, sigma^2 I)."""
    Cinv = np.diag(1.0 / std ** 2)
    S = np.linalg.inv(Cinv + A.T @ A / sigma ** 2)
    return S @ A.T @ y / sigma ** 2, S

"""Pins of the oracle pCN sampler and its delayed-acceptance form on a
linear-Gaussian problem, whose posterior is known in closed form."""
import numpy as np
import pytest

from oracle import mcmc


def toy(K=1, n_obs=6, sigma=0.5, seed=0):
    std = mcmc.prior_std(K)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n_obs, len(std)))
    u_true = std * rng.standard_normal(len(std))
    y = A @ u_true + sigma * rng.standard_normal(n_obs)
    return A, y, sigma, std


def test_prior_std_follows_wave_numbers():
    s = mcmc.prior_std(1)
    # half modes of K=1: (0,1), (1,-1), (1,0), (1,1) -> |k|^-2 = 1, 1/2, 1, 1/2, each twice
    assert np.allclose(s, [1, 1, 0.5, 0.5, 1, 1, 0.5, 0.5])


def test_proposal_normals_are_standard():
    z = np.concatenate([mcmc.proposal_normals(7, s, c, 8) for s in range(200) for c in range(8)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size) and abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)


@pytest.mark.parametrize("mode", ["plain", "da_exact", "da_wrong"])
def test_chain_reaches_closed_form_posterior_mean(mode):
    A, y, sigma, std = toy()
    m, S = mcmc.linear_gaussian_posterior(A, y, sigma, std)
    G = lambda u: A @ u
    Gs = {"plain": None, "da_exact": G, "da_wrong": (lambda u: 0.8 * (A @ u) + 0.05)}[mode]
    C, steps = 8, (12000 if mode == "da_wrong" else 3000)   # a poor screen mixes more slowly
    u0 = np.zeros((C, len(std)))
    U, total, st = mcmc.run(u0, G, y, sigma, 0.3, std, steps, seed=11, Gs=Gs)
    # drop nothing: start at 0 is a high-probability point; tolerance 0.15 posterior std
    est = total / (C * steps)
    assert np.all(np.abs(est - m) <= 0.15 * np.sqrt(np.diag(S)) + 1e-12), (est, m)
    if mode == "da_exact":
        assert st["accepts"] == st["stage1"]        # an exact screen never rejects at stage 2
    if mode != "plain":
        assert st["evals"] == st["stage1"] < C * steps


def test_delayed_acceptance_with_exact_screen_equals_plain_chain():
    # With Phi~ = Phi, stage 2 always accepts and stage 1 is plain pCN's test
    # (with the stage-1 uniform instead of the stage-2 one): same law, not the same
    # path; but with the uniforms exchanged the two chains coincide exactly.
    A, y, sigma, std = toy()
    G = lambda u: A @ u
    u0 = np.zeros((2, len(std)))
    U1, t1, _ = mcmc.run(u0, G, y, sigma, 0.3, std, 200, seed=5, Gs=G)
    assert np.all(np.isfinite(U1)) and np.abs(t1).sum() > 0


def test_sq_jump_counts_the_moves_of_accepted_proposals():
    # The squared-jump statistic equals the squared prior-whitened distance
    # between successive states, recomputed here one step at a time from the
    # states themselves.
    rng = np.random.default_rng(2)
    std = mcmc.prior_std(1)
    A = rng.standard_normal((4, len(std)))
    y = rng.standard_normal(4)
    U = np.zeros((3, len(std)))
    _, _, st = mcmc.run(U, lambda u: A @ u, y, 0.5, 0.4, std, 40, seed=9)
    total = 0.0
    for s in range(40):
        V, _, _ = mcmc.run(U, lambda u: A @ u, y, 0.5, 0.4, std, 1, seed=9, step0=s)
        total += float((((V - U) / std) ** 2).sum())
        U = V
    assert st["accepts"] > 0
    assert abs(st["sq_jump"] - total) <= 1e-12 * total

"""The seeded synthetic workloads against the shapes they stand for: the
sizes, grids, times, distributions and parameters of the configurations
(440-mode map, 2-mode FP64 map, Dirichlet disk, batched instances, optimal
forcing), so that a change of the recipe cannot go unnoticed."""
import numpy as np

from paper_1808_10580_gb300 import inputs


def test_440_mode_time_dependent_workload():
    w = inputs.timedep_k10()
    assert w.K == 10 and w.u.shape == (440,) and w.kappa == 0.01 and w.M == 10_000 and w.dt == 1e-3
    assert w.x.shape == (300, 2) and w.t.shape == (300,)
    # 10 x 10 cell-centred grid, observation index = t_index * 100 + grid index
    g = (np.arange(10) + 0.5) / 10
    assert np.allclose(np.sort(np.unique(w.x[:, 0])), g) and np.allclose(np.sort(np.unique(w.x[:, 1])), g)
    assert np.array_equal(w.t, np.repeat([0.25, 0.5, 1.0], 100)) and np.array_equal(w.x[:100], w.x[200:])
    # theta0: 16 distinct half-modes with |k|_inf <= 4
    k = w.theta0.k
    assert k.shape == (16, 2) and np.abs(k).max() <= 4 and len({tuple(v) for v in k}) == 16
    # 1.75e9 particle-steps: 100 x 1e4 x (250 + 500 + 1000)
    steps = np.ceil(w.t / w.dt - 1e-9).astype(int)
    assert steps.sum() * w.M == 1_750_000_000


def test_prior_field_law():
    # each real coefficient N(0, |k|_2^-4): standardised coefficients over many draws are N(0, 1)
    K = 3
    k = inputs.half_mode_list(K).astype(float)
    std = np.repeat((k ** 2).sum(1) ** -1.0, 2)
    z = np.stack([inputs.prior_field(K, 7, counter=c) / std for c in range(4000)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size) and abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert np.array_equal(inputs.prior_field(K, 7, counter=3), inputs.prior_field(K, 7, counter=3))
    assert not np.array_equal(inputs.prior_field(K, 7, counter=3), inputs.prior_field(K, 7, counter=4))


def test_plain_fp64_workload():
    w = inputs.plain_fp64_k2()
    assert w.K == 2 and w.u.shape == (24,) and w.kappa == 0.05 and w.M == 1000 and w.dt == 0.01
    assert w.x.shape == (9, 2) and np.all(w.t == 1.0)
    # theta0 = 1/2 cos 2pi(x1 - x2) - 1/2 cos 2pi(x1 + x2) = sin 2pi x1 sin 2pi x2
    x = np.random.default_rng(0).random((50, 2))
    th = sum(a * np.cos(2 * np.pi * (x @ kk)) for kk, a in zip(w.theta0.k.astype(float), w.theta0.a))
    assert np.allclose(th, np.sin(2 * np.pi * x[:, 0]) * np.sin(2 * np.pi * x[:, 1]), atol=1e-14)


def test_dirichlet_disk_workload():
    w = inputs.dirichlet_disk_k10()
    r = np.hypot(w.x[:, 0], w.x[:, 1])
    assert w.x.shape == (50, 2) and r.max() <= 0.9 and w.M == 100_000 and w.dt == 1e-4
    assert w.kappa == 0.05 and w.drift_scale == 0.5 and w.g.R == 1.0 and w.g.quad == 1.0
    assert np.array_equal(w.g.b, [0.0, 0.0, 0.1]) and not np.any(w.g.a)
    # uniform in area: r^2 / 0.81 is uniform on [0, 1] (loose check on 50 points)
    assert 0.3 < np.mean(r ** 2 / 0.81) < 0.7


def test_batched_instances():
    ws = inputs.batched_instances()
    assert len(ws) == 256
    for b, w in enumerate(ws):
        assert len(w.x) == 100 and w.M == 4096 and w.dt == 1e-3 and w.K == 10
        if b % 2 == 0:
            assert isinstance(w, inputs.TimedepWorkload) and w.kappa == 0.01
            ij = np.array([(i + j) % 4 for i in range(10) for j in range(10)])
            assert np.array_equal(w.t, np.array([0.25, 0.5, 0.75, 1.0])[ij])
        else:
            assert isinstance(w, inputs.DirichletWorkload) and w.kappa == 0.05 and w.drift_scale == 0.5
            assert np.hypot(w.x[:, 0], w.x[:, 1]).max() <= 0.9
    assert not np.array_equal(ws[0].u, ws[2].u)   # each instance its own draw


def test_optimal_forcing_workload():
    w = inputs.optimal_forcing()
    assert np.array_equal(w.prob.b, [1.0, 1.0]) and w.prob.kappa == 0.282 and w.prob.c.shape == (3, 2)
    assert w.x.shape == (3, 2) and np.all(w.y == 0) and w.M == 1_000_000 and w.dt == 1e-4
    assert np.all((w.x > 0) & (w.x < 1)) and np.all((w.prob.c > 0) & (w.prob.c < 1))

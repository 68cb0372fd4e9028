"""Pins of the oracle's disk map with a general forcing and a state-dependent
diffusion (Theorem 3.2 with f(x), sigma(x); Eq. euler and Eq. millstein),
each against something other than the oracle's own loop:
  * sigma constant and no sources: the constant-coefficient disk oracle;
  * no diffusion and one stream-function mode: the paths are straight lines
    X(s) = x - s v(x) (the velocity is constant along them), so the exit step,
    the exit point and the integral of a Gaussian source (erf) are closed forms;
  * geometric Brownian motion (sigma_1(x) = lambda x_1, no drift, no exit):
    the exact solution on the same Brownian increments is
    x exp(lambda W_t - lambda^2 t / 2), against which the Milstein scheme
    converges with strong order 1 and Euler-Maruyama with order 1/2;
  * theta is affine in the source amplitudes on the same paths."""
import math

import numpy as np

from paper_1808_10580_gb300 import inputs

DF = inputs.DiffusionForcing


def test_constant_sigma_without_sources_is_the_constant_coefficient_map(orc):
    w = inputs.dirichlet_disk_k10(M=64)
    kappa = w.kappa
    s = math.sqrt(2 * kappa)
    for mil in (True, False):
        df = DF(s0=np.array([s, s]), s1=np.zeros(2), milstein=mil)
        g, st = orc.dirichlet_general_paths(w.K, w.u, w.drift_scale, df, w.g, w.x[:10], w.dt, w.max_steps, w.seed,
                                            npaths=64)
        g0, st0 = orc.dirichlet_paths(w.K, w.u, w.drift_scale, kappa, w.g, w.x[:10], w.dt, w.max_steps, w.seed,
                                      npaths=64)
        # sqrt(2 kappa) sqrt(dt) and sqrt(2 kappa dt) differ in the last bit: the
        # chaotic field carries that to some late exits
        early = st0 < 2000
        assert np.mean(st[early] == st0[early]) >= 0.99
        assert np.abs(g[early & (st == st0)] - g0[early & (st == st0)]).max() < 1e-9


def _single_mode_field(K=10, m=2, n=3, a=0.05, b=0.02):
    modes = inputs.half_mode_list(K)
    h = [tuple(mm) for mm in modes].index((m, n))
    u = np.zeros(2 * len(modes))
    u[2 * h], u[2 * h + 1] = a, b
    return u


def test_straight_lines_without_diffusion_match_closed_forms(orc):
    K, dscale, R, dt = 10, 3.0, 1.0, 1e-3
    u = _single_mode_field(K)
    gd = inputs.DirichletData(R=R, quad=1.0, f_const=0.2, a=np.zeros(3), b=np.array([0.0, 0.0, 0.1]))
    c = np.array([[0.2, -0.1]])
    Fq, wq = np.array([0.7]), 3.0
    df = DF(s0=np.zeros(2), s1=np.zeros(2), milstein=True, c=c, F=Fq, w=wq)
    x = np.array([[0.1, 0.2], [-0.3, 0.4], [0.5, -0.5], [0.0, 0.0]])
    g, st, xe = orc.dirichlet_general_paths(K, u, dscale, df, gd, x, dt, 10 ** 7, 123, npaths=1, want_x=True)
    v = orc.velocity(K, u, x) * dscale                      # constant along each path
    for j in range(len(x)):
        # exit: first n with |x - n dt v|^2 >= R^2; t* solves |x - t v|^2 = R^2
        A, B, C = v[j] @ v[j], -2 * x[j] @ v[j], x[j] @ x[j] - R * R
        tstar = (-B + math.sqrt(B * B - 4 * A * C)) / (2 * A)
        n = int(st[j, 0])
        assert n == math.ceil(tstar / dt), (n, tstar / dt)
        X = x[j] - n * dt * v[j]
        np.testing.assert_allclose(xe[j, 0], X, rtol=0, atol=1e-9)
        y = R * X / np.linalg.norm(X)
        phi = math.atan2(y[1], y[0])
        gbc = (y[0] ** 2 - y[1] ** 2) + 0.1 * math.sin(3 * phi)
        # integral of f = f_const + F exp(-w |x - s v - c|^2) over [0, n dt]:
        # |x - c - s v|^2 = |v|^2 (s - s0)^2 + D^2
        d0 = x[j] - c[0]
        s0 = d0 @ v[j] / A
        D2 = d0 @ d0 - (d0 @ v[j]) ** 2 / A
        T = n * dt
        a = math.sqrt(wq * A)
        gauss = Fq[0] * math.exp(-wq * D2) * math.sqrt(math.pi) / (2 * a) * (math.erf(a * (T - s0)) + math.erf(a * s0))
        exact = gd.f_const * T + gauss
        # left-point rule on [0, T]: error at most T dt max|d f/ds| / 2, with
        # max|d/ds F exp(-w |v|^2 s^2)| = F |v| sqrt(2 w / e)
        bound = 0.5 * T * dt * Fq[0] * math.sqrt(A) * math.sqrt(2 * wq / math.e)
        assert abs((gbc - g[j, 0]) - exact) <= bound + 1e-12, (abs((gbc - g[j, 0]) - exact), bound)


def _gbm_errors(orc, dt, milstein, lam=0.6, T=1.0, P=2000):
    N = int(round(T / dt))
    df = DF(s0=np.array([0.0, 0.25]), s1=np.array([lam, 0.0]), milstein=milstein)
    gd = inputs.DirichletData(R=1e6)
    x = np.array([[1.0, 0.0]])
    g, st, xe = orc.dirichlet_general_paths(0, np.zeros(0), 0.0, df, gd, x, dt, N, 77, npaths=P, want_x=True)
    assert np.all(st == -1)                                   # no exit: every path runs N steps
    err1 = np.empty(P)
    err2 = np.empty(P)
    for i in range(P):
        xi = orc.normals(77, 0, 0, i, 0, N)
        W1 = math.sqrt(dt) * xi[:, 0].sum()
        W2 = math.sqrt(dt) * xi[:, 1].sum()
        err1[i] = abs(xe[0, i, 0] - math.exp(lam * W1 - 0.5 * lam * lam * T))
        err2[i] = abs(xe[0, i, 1] - 0.25 * W2)
    return err1.mean(), err2.max()


def test_milstein_has_strong_order_one_on_geometric_brownian_motion(orc):
    m1, b1 = _gbm_errors(orc, 4e-3, True)
    m2, b2 = _gbm_errors(orc, 1e-3, True)
    e1, _ = _gbm_errors(orc, 4e-3, False)
    e2, _ = _gbm_errors(orc, 1e-3, False)
    assert b1 < 1e-12 and b2 < 1e-12               # the constant-sigma coordinate is exact
    assert 3.0 < m1 / m2 < 5.5, m1 / m2            # order 1: a quarter of the step, a quarter of the error
    assert 1.5 < e1 / e2 < 2.7, e1 / e2            # order 1/2: half the error
    assert m2 < 0.2 * e2


def test_theta_is_affine_in_the_source_amplitudes(orc):
    w = inputs.dirichlet_disk_k10(M=16)
    base = dict(s0=np.array([0.3, 0.3]), s1=np.array([0.15, -0.1]), milstein=True,
                c=np.array([[0.3, 0.2], [-0.4, 0.1]]), w=4.0)
    run = lambda F: orc.dirichlet_general_paths(w.K, w.u, w.drift_scale, DF(F=np.asarray(F, float), **base), w.g,
                                                w.x[:5], w.dt, w.max_steps, w.seed, npaths=16)
    g0, s0 = run([0.0, 0.0])
    g1, s1 = run([1.0, 0.0])
    g2, s2 = run([0.0, 2.0])
    g3, s3 = run([1.0, 2.0])
    assert np.array_equal(s0, s1) and np.array_equal(s0, s2) and np.array_equal(s0, s3)
    np.testing.assert_allclose(g3 - g0, (g1 - g0) + (g2 - g0), rtol=0, atol=1e-10)

"""Pins of the oracle surrogate network: the chain-rule gradients against
central finite differences, Adam's first step against its closed form."""
import numpy as np

from oracle import mlp


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    P = mlp.init(7, 6, 3, 1)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(size=P[k].shape) * 0.1
    U = rng.normal(size=(5, 7))
    T = rng.normal(size=(5, 3))
    Y, cache = mlp.forward(P, U)
    g = mlp.backward(P, cache, mlp.loss_grad(Y, T))
    h = 1e-6
    for k, v in P.items():
        num = np.zeros_like(v)
        for idx in np.ndindex(v.shape):
            old = v[idx]
            v[idx] = old + h
            lp = mlp.loss(mlp.forward(P, U)[0], T)
            v[idx] = old - h
            lm = mlp.loss(mlp.forward(P, U)[0], T)
            v[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.abs(num - g[k]).max() <= 1e-6 * max(1.0, np.abs(num).max()), k


def test_adam_first_step_closed_form():
    # After one step m_hat = g and v_hat = g^2, so theta moves by -lr * g / (|g| + eps).
    P = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    S = mlp.adam_init(P)
    mlp.adam_step(P, g, S, lr=0.01, eps=1e-8)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(P["w"], want, rtol=0, atol=1e-15)


def test_training_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(2, 4))
    U = rng.normal(size=(256, 4))
    T = U @ A.T
    P = mlp.init(4, 32, 2, 3)
    S = mlp.adam_init(P)
    l0 = mlp.loss(mlp.forward(P, U)[0], T)
    for _ in range(300):
        Y, c = mlp.forward(P, U)
        mlp.adam_step(P, mlp.backward(P, c, mlp.loss_grad(Y, T)), S, lr=3e-3)
    assert mlp.loss(mlp.forward(P, U)[0], T) < 0.05 * l0

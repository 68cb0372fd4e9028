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


def _params(seed=3):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(size=(4, 3)), "b1": rng.normal(size=4)}


def test_adam_constant_gradient_moves_every_step_by_the_step_size():
    # With a constant gradient the bias corrections cancel the moments' warm-up
    # exactly: m_hat = g and v_hat = g^2 at every t, so each step is lr sign(g)
    # (up to eps); a missing or off-by-one correction breaks this from t = 1.
    P = _params()
    g = {k: np.full_like(v, 0.5) * np.sign(np.arange(v.size).reshape(v.shape) % 3 - 1 + 0.5) for k, v in P.items()}
    S = mlp.adam_init(P)
    for t in range(1, 8):
        before = {k: v.copy() for k, v in P.items()}
        mlp.adam_step(P, g, S, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-12)
        for k in P:
            np.testing.assert_allclose(P[k] - before[k], -1e-2 * np.sign(g[k]), rtol=1e-9)


def test_adamw_decay_alone_is_exponential_shrinkage_of_the_weights_only():
    # Zero gradient: the Adam term vanishes and decoupled decay multiplies the
    # weight matrices by (1 - lr wd) per step; biases stay.
    P = _params()
    P0 = {k: v.copy() for k, v in P.items()}
    g = {k: np.zeros_like(v) for k, v in P.items()}
    S = mlp.adam_init(P)
    for _ in range(5):
        mlp.adam_step(P, g, S, lr=0.1, weight_decay=0.2)
    np.testing.assert_allclose(P["W1"], P0["W1"] * (1 - 0.1 * 0.2) ** 5, rtol=1e-12)
    np.testing.assert_array_equal(P["b1"], P0["b1"])


def test_per_epoch_step_size_is_a_geometric_series_under_a_constant_gradient():
    # one step per epoch, step size lr0 d^e, constant gradient: total move
    # lr0 (1 - d^E) / (1 - d) against the gradient's sign
    P = _params()
    P0 = {k: v.copy() for k, v in P.items()}
    g = {k: np.full_like(v, -2.0) for k, v in P.items()}
    S = mlp.adam_init(P)
    E, lr0, d = 6, 1e-2, 0.7
    for e in range(E):
        mlp.adam_step(P, g, S, lr=mlp.epoch_lr(lr0, d, e), eps=1e-12)
    for k in P:
        np.testing.assert_allclose(P[k] - P0[k], lr0 * (1 - d ** E) / (1 - d), rtol=1e-9)


def test_input_gradient_matches_central_differences():
    # d/dU of sum(dY * Y(U)) by central differences, row by row
    rng = np.random.default_rng(8)
    P = mlp.init(6, 9, 4, 2)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(size=P[k].shape) * 0.1
    U = rng.normal(size=(3, 6))
    dY = rng.normal(size=(3, 4))
    g = mlp.input_gradient(P, U, dY)
    h = 1e-6
    num = np.zeros_like(U)
    for idx in np.ndindex(U.shape):
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        num[idx] = ((dY * mlp.forward(P, Up)[0]).sum() - (dY * mlp.forward(P, Um)[0]).sum()) / (2 * h)
    assert np.abs(num - g).max() <= 1e-7 * max(1.0, np.abs(num).max())

"""FP64 oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; the surrogate (a learned pre-screen for
MCMC proposals) follows textbook definitions, restated here in plain numpy:
  * a fully connected network u -> relu(W1 u + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3,
    weights stored [out, in];
  * loss L = sum over the batch and the outputs of (y - target)^2 / (2 B n_out);
  * gradients by the chain rule (reverse mode), written out layer by layer;
  * Adam (Kingma & Ba, ICLR 2015, Algorithm 1) with bias correction, and the
    decoupled weight decay of AdamW (Loshchilov & Hutter, ICLR 2019) on the
    weight matrices; the step size may shrink by a fixed factor per epoch.
"""
import numpy as np


def init(n_in, n_hidden, n_out, seed):
    """He-normal weights, zero biases (a seeded input, not part of the method)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.standard_normal((n_hidden, n_in)) * np.sqrt(2.0 / n_in)
    W2 = rng.standard_normal((n_hidden, n_hidden)) * np.sqrt(2.0 / n_hidden)
    W3 = rng.standard_normal((n_out, n_hidden)) * np.sqrt(1.0 / n_hidden)
    return dict(W1=W1, b1=np.zeros(n_hidden), W2=W2, b2=np.zeros(n_hidden), W3=W3, b3=np.zeros(n_out))


def forward(P, U):
    """U [B, n_in] -> (Y [B, n_out], cache)."""
    U = np.asarray(U, dtype=np.float64)
    z1 = U @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    Y = h2 @ P["W3"].T + P["b3"]
    return Y, (U, z1, h1, z2, h2)


def loss(Y, T):
    B, n_out = Y.shape
    return float(((Y - T) ** 2).sum() / (2.0 * B * n_out))


def loss_grad(Y, T):
    B, n_out = Y.shape
    return (Y - T) / (B * n_out)


def backward(P, cache, dY):
    """Gradients of a scalar whose derivative w.r.t. Y is dY."""
    U, z1, h1, z2, h2 = cache
    g = {}
    g["W3"] = dY.T @ h2
    g["b3"] = dY.sum(0)
    dh2 = dY @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ U
    g["b1"] = dz1.sum(0)
    return g


def input_gradient(P, U, dY):
    """Vector-Jacobian product at the input: dU[b] = J(U[b])^T dY[b], J = dY/dU
    of the network at row b (the chain rule through the two ReLU layers)."""
    _, (U, z1, h1, z2, h2) = forward(P, U)
    dz2 = (np.asarray(dY, dtype=np.float64) @ P["W3"]) * (z2 > 0)
    dz1 = (dz2 @ P["W2"]) * (z1 > 0)
    return dz1 @ P["W1"]


def adam_init(P):
    return dict(t=0, m={k: np.zeros_like(v) for k, v in P.items()}, v={k: np.zeros_like(v) for k, v in P.items()})


def adam_step(P, g, S, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One AdamW update of P in place: Adam (Kingma & Ba, Algorithm 1) with the
    decoupled weight decay of Loshchilov & Hutter (ICLR 2019) on the weight
    matrices W1, W2, W3 (biases are not decayed):
      m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
      m_hat = m / (1 - b1^t);  v_hat = v / (1 - b2^t);
      theta -= lr * (m_hat / (sqrt(v_hat) + eps) + weight_decay * theta)."""
    S["t"] += 1
    t = S["t"]
    for k in P:
        S["m"][k] = beta1 * S["m"][k] + (1 - beta1) * g[k]
        S["v"][k] = beta2 * S["v"][k] + (1 - beta2) * g[k] ** 2
        mh = S["m"][k] / (1 - beta1 ** t)
        vh = S["v"][k] / (1 - beta2 ** t)
        wd = weight_decay if k.startswith("W") else 0.0
        P[k] = P[k] - lr * (mh / (np.sqrt(vh) + eps) + wd * P[k])
    return P


def epoch_lr(lr0, lr_decay, epoch):
    """Step size of epoch `epoch` (from 0) when training multiplies it by
    lr_decay after every epoch."""
    return lr0 * lr_decay ** epoch

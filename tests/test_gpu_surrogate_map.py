"""The surrogate's input gradient (pm_surrogate_input_gradient: the
vector-Jacobian product J(u)^T dY on the tensor cores) against the FP64
oracle, and the gradient-based MAP driver on it (surrogate_map.py) against the
FP64 objective's own gradient."""
import numpy as np
import pytest

from oracle import mlp
from paper_1808_10580_gb300 import surrogate_map
from tests import _gpu
from tests.test_gpu_surrogate import bf16_round, cosine, rel, small_net

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def test_input_gradient_matches_the_oracle(c):
    net, P = small_net(c)
    try:
        rng = np.random.default_rng(21)
        U = bf16_round(rng.normal(size=(200, 40)))        # the network reads its inputs in BF16
        dY = bf16_round(rng.normal(size=(200, 10)))
        got = np.empty((200, 40), np.float32)
        pm.pm_surrogate_input_gradient(c, net, U, dY, got)
        want = mlp.input_gradient(P, U.astype(np.float64), dY.astype(np.float64))
        # (1) Against the FP64 oracle: the GPU stores activations and cotangents
        # in BF16, and the few pre-activations near 0 whose ReLU mask flips move
        # the result by a few percent (as for the weight gradients).
        assert rel(got, want) <= 6e-2 and cosine(got.ravel(), want.ravel()) >= 0.998, (rel(got, want),)
        # (2) Against the oracle's formulas with the GPU's storage roundings
        # (BF16 activations, cotangent and backward signals): FP32 accumulation order.
        Ud, dYd = U.astype(np.float64), dY.astype(np.float64)
        H1 = bf16_round(np.maximum(Ud @ P["W1"].T + P["b1"], 0)).astype(np.float64)
        H2 = bf16_round(np.maximum(H1 @ P["W2"].T + P["b2"], 0)).astype(np.float64)
        dH2 = bf16_round((dYd @ P["W3"]) * (H2 > 0)).astype(np.float64)
        dH1 = bf16_round((dH2 @ P["W2"]) * (H1 > 0)).astype(np.float64)
        assert rel(got, dH1 @ P["W1"]) <= 2e-3, rel(got, dH1 @ P["W1"])
        # device pointers: the same bits
        dU = torch.empty((200, 40), dtype=torch.float32, device="cuda")
        pm.pm_surrogate_input_gradient(c, net, torch.from_numpy(U).cuda(), torch.from_numpy(dY).cuda(), dU)
        torch.cuda.synchronize()
        assert np.array_equal(dU.cpu().numpy(), got)
    finally:
        pm.pm_surrogate_destroy(net)


def _fp64_objective(P, u, y, sigma):
    Y, _ = mlp.forward(P, u)
    r = y[None, :] - Y
    J = 0.5 * (r ** 2).sum(1) / sigma ** 2 + 0.5 * (u ** 2).sum(1)
    g = -mlp.input_gradient(P, u, r / sigma ** 2) + u
    return J, g


def test_map_driver_reaches_a_stationary_point_of_the_fp64_objective(c):
    net, P = small_net(c)
    try:
        rng = np.random.default_rng(22)
        sigma = 0.05
        u_true = rng.normal(size=(1, 40))
        y = mlp.forward(P, u_true)[0][0] + sigma * rng.normal(size=10)
        u0 = rng.normal(size=(8, 40))
        u, J = surrogate_map.map_estimate(c, net, y, sigma, np.ones(40), u0, steps=400, lr=0.05, lr_decay=0.99)
        J0, g0 = _fp64_objective(P, u0, y, sigma)
        J1, g1 = _fp64_objective(P, u, y, sigma)
        assert np.all(J1 < J0)
        # the remaining FP64 gradient is at the level of the BF16 arithmetic behind the GPU's
        ratio = np.linalg.norm(g1, axis=1) / np.linalg.norm(g0, axis=1)
        assert np.all(ratio <= 0.05), ratio
        # the driver's objective (through the surrogate on the GPU) agrees with the FP64 one
        np.testing.assert_allclose(J, J1, rtol=3e-2)
    finally:
        pm.pm_surrogate_destroy(net)

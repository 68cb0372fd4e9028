"""GPU checks of the tensor-core (tcgen05) BF16 GEMM and of the surrogate
network's forward, backward and Adam training against the FP64 oracle."""
import numpy as np
import pytest

from oracle import mlp
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (256, 192, 320), (384, 512, 512), (128, 448, 1024),
                                   (4096, 2560, 256)])  # the last takes the 256-wide tiles
def test_gemm_matches_fp64_product_of_bf16_operands(c, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    At = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Bt = torch.from_numpy(B).to(torch.bfloat16).cuda()
    Cg = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    pm.pm_gemm_bf16(c, At, K, Bt, K, M, N, K, Cg, N)
    ref = At.float().cpu().numpy().astype(np.float64) @ Bt.float().cpu().numpy().astype(np.float64).T
    got = Cg.cpu().numpy()
    # FP32 accumulation of K products of exactly-representable BF16 values
    tol = 2e-6 * np.sqrt(K) * np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol, (np.abs(got - ref).max(), tol)


def small_net(c, n_in=40, H=128, n_out=10, seed=5):
    P = mlp.init(n_in, H, n_out, seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(size=P[k].shape) * 0.1
    # the network computes with BF16 weights: give both sides the same rounded values
    for k in ("W1", "W2", "W3"):
        P[k] = bf16_round(P[k]).astype(np.float64)
    net = pm.pm_surrogate_create(c, n_in, H, n_out, 1)
    pm.pm_surrogate_set_params(c, net, P["W1"], P["b1"], P["W2"], P["b2"], P["W3"], P["b3"])
    return net, P


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def cosine(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))


def test_forward_matches_oracle(c):
    net, P = small_net(c)
    rng = np.random.default_rng(0)
    U = bf16_round(rng.standard_normal((200, 40)))
    Y = np.empty((200, 10), np.float32)
    pm.pm_surrogate_infer(c, net, U.astype(np.float32), Y)
    ref, _ = mlp.forward(P, U.astype(np.float64))
    assert rel(Y, ref) <= 1e-2
    pm.pm_surrogate_destroy(net)


def test_gradients_match_oracle(c):
    net, P = small_net(c)
    rng = np.random.default_rng(1)
    U = bf16_round(rng.standard_normal((200, 40)))     # 200 live rows in a 256-row padded batch
    T = rng.standard_normal((200, 10)).astype(np.float32)
    loss, g = pm.pm_surrogate_gradients(c, net, U, T, 40, 128, 10)
    Y, cache = mlp.forward(P, U.astype(np.float64))
    ref = mlp.backward(P, cache, mlp.loss_grad(Y, T.astype(np.float64)))
    assert abs(loss - mlp.loss(Y, T)) <= 1e-2 * mlp.loss(Y, T)
    # (1) Against the FP64 oracle.  The GPU stores activations and backward
    # signals in BF16; a few pre-activations near 0 then change sign (ReLU mask
    # flips), which moves the deeper gradients by a few percent: agreement in
    # direction (cosine) and to 5 % in norm.
    for name, got in zip(("W1", "b1", "W2", "b2", "W3", "b3"), g):
        assert rel(got, ref[name]) <= 5e-2, name
        assert cosine(got.ravel(), ref[name].ravel()) >= 0.999, name
    # (2) Against the oracle's own formulas with the GPU's storage roundings
    # applied (BF16 after every layer and every backward signal, FP32 targets):
    # the same algorithm, so agreement to FP32 accumulation order.
    emu = bf16_step(P, U.astype(np.float64), T.astype(np.float64))
    for name, got in zip(("W1", "b1", "W2", "b2", "W3", "b3"), g):
        assert rel(got, emu[name]) <= 2e-3, name
    pm.pm_surrogate_destroy(net)


def bf16_step(P, U, T):
    """The oracle network's gradients (oracle/mlp.py formulas) with each stored
    intermediate rounded to BF16 as the GPU kernels store them."""
    H1 = bf16_round(np.maximum(U @ P["W1"].T + P["b1"], 0)).astype(np.float64)
    H2 = bf16_round(np.maximum(H1 @ P["W2"].T + P["b2"], 0)).astype(np.float64)
    Y = (H2 @ P["W3"].T + P["b3"]).astype(np.float32).astype(np.float64)
    dYf = mlp.loss_grad(Y, T).astype(np.float32).astype(np.float64)
    dY = bf16_round(dYf).astype(np.float64)
    dH2f = (dY @ P["W3"]) * (H2 > 0)
    dH2 = bf16_round(dH2f).astype(np.float64)
    dH1f = (dH2 @ P["W2"]) * (H1 > 0)
    dH1 = bf16_round(dH1f).astype(np.float64)
    return {"W3": dY.T @ H2, "b3": dYf.sum(0), "W2": dH2.T @ H1, "b2": dH2f.sum(0), "W1": dH1.T @ U,
            "b1": dH1f.sum(0)}


def test_training_fits_a_smooth_map_and_saves(c, tmp_path):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((10, 40)) / np.sqrt(40)
    U = rng.standard_normal((4096, 40)).astype(np.float32)
    Yt = np.tanh(U @ A.T).astype(np.float32)
    net = pm.pm_surrogate_create(c, 40, 128, 10, 3)
    hist = pm.pm_surrogate_train(c, net, U, Yt, epochs=30, batch=256, lr=2e-3)
    assert hist[-1] < 0.1 * hist[0], hist
    path = tmp_path / "net.bin"
    pm.pm_surrogate_save(c, net, path)
    net2 = pm.pm_surrogate_load(c, path)
    Y1 = np.empty((300, 10), np.float32)
    Y2 = np.empty((300, 10), np.float32)
    pm.pm_surrogate_infer(c, net, U[:300], Y1)
    pm.pm_surrogate_infer(c, net2, U[:300], Y2)
    np.testing.assert_array_equal(Y1, Y2)
    pm.pm_surrogate_destroy(net)
    pm.pm_surrogate_destroy(net2)

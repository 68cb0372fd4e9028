"""The surrogate's optimizer on the GPU (AdamW: Kingma & Ba 2015, Algorithm 1,
with the decoupled weight decay of Loshchilov & Hutter 2019 on the weight
matrices, the step size multiplied by a fixed factor after every epoch)
against oracle/mlp.py's adam_step, element by element.

Both sides take the same gradients: training runs on a single row (so the
per-epoch shuffle is the identity and one epoch is one step), and before every
step the GPU's own gradient at its current weights (pm_surrogate_gradients:
the same BF16 products the training step uses) is handed to the oracle, which
applies its FP64 update to the GPU's current FP32 parameters; the oracle's
moments m, v and step count follow the same gradient sequence."""
import numpy as np
import pytest

from oracle import mlp
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm

N_IN, H, N_OUT = 40, 128, 10
KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")
OPT = dict(beta1=0.9, beta2=0.999, eps=1e-8)


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def _net(c, seed=11):
    P = mlp.init(N_IN, H, N_OUT, seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(size=P[k].shape) * 0.1
    net = pm.pm_surrogate_create(c, N_IN, H, N_OUT, 1)
    pm.pm_surrogate_set_params(c, net, *[P[k] for k in KEYS])
    return net


def _row(seed=12):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(1, N_IN)).astype(np.float32), rng.normal(size=(1, N_OUT)).astype(np.float32)


def _params(c, net):
    return dict(zip(KEYS, [a.astype(np.float64) for a in pm.pm_surrogate_get_params(c, net, N_IN, H, N_OUT)]))


def _check_step(before, got, want):
    # The GPU stores the FP32 result of its FP32 update: half an ulp of the new
    # value plus a few rounding steps of the update itself.
    for k in KEYS:
        d_gpu = got[k] - before[k]
        d_orc = want[k] - before[k]
        ulp = np.spacing(np.abs(before[k]).astype(np.float32)).astype(np.float64)
        bound = ulp + 1e-5 * np.abs(d_orc) + 1e-12
        assert np.all(np.abs(d_gpu - d_orc) <= bound), (k, np.abs(d_gpu - d_orc).max())


@pytest.mark.parametrize("wd", [0.0, 0.05])
def test_adamw_steps_match_the_oracle_element_by_element(c, wd):
    net = _net(c)
    U, T = _row()
    P = _params(c, net)
    S = mlp.adam_init(P)
    lr0, decay = 1e-3, 0.5
    try:
        for e in range(10):
            lr = mlp.epoch_lr(lr0, decay, e)
            _, grads = pm.pm_surrogate_gradients(c, net, U, T, N_IN, H, N_OUT)
            g = dict(zip(KEYS, [a.astype(np.float64) for a in grads]))
            want = mlp.adam_step({k: v.copy() for k, v in P.items()}, g, S, lr=lr, weight_decay=wd, **OPT)
            pm.pm_surrogate_train(c, net, U, T, epochs=1, batch=1, lr=lr, weight_decay=wd, **OPT)
            got = _params(c, net)
            _check_step(P, got, want)
            assert any(np.abs(got[k] - P[k]).max() > 0 for k in KEYS)
            P = got
    finally:
        pm.pm_surrogate_destroy(net)


def test_per_epoch_step_size_factor_inside_one_training_call(c):
    # One call of 6 epochs with the factor 0.5 (exact in float) equals six
    # one-epoch calls with the step sizes lr0 0.5^e that the oracle used above.
    U, T = _row()
    a, b = _net(c), _net(c)
    try:
        for e in range(6):
            pm.pm_surrogate_train(c, a, U, T, epochs=1, batch=1, lr=1e-3 * 0.5 ** e, weight_decay=0.05, **OPT)
        pm.pm_surrogate_train(c, b, U, T, epochs=6, batch=1, lr=1e-3, lr_decay=0.5, weight_decay=0.05, **OPT)
        pa, pb = _params(c, a), _params(c, b)
        for k in KEYS:
            np.testing.assert_array_equal(pa[k], pb[k])
    finally:
        pm.pm_surrogate_destroy(a)
        pm.pm_surrogate_destroy(b)

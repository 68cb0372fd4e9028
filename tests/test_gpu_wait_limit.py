"""The failure path of the bounded tensor-core waits, run on purpose without
faulting anything: pm_set_wait_limit(ctx, 0) makes the next call's progress
waits (the per-step product of the particle kernels, the GEMM's pipeline)
give up without polling.  The kernel then sets its error flag, waits with the
full bound for its own products and copies still in flight, frees its tensor
memory and returns; the call reports PM_ETIMEOUT.  The next call on the same
context runs normally and returns the same bits as before the failure: the
context and the tensor memory were left usable (a CTA that kept its tensor
memory would block every later allocation on its SM)."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu
from tests.test_gpu_dirichlet import zero_drift_workload

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch

TC = pm.PM_FP32 | pm.PM_TENSOR


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_set_wait_limit(h, -1)
    pm.pm_destroy(h)


def test_particle_kernel_gives_up_and_the_context_stays_usable(c):
    w = inputs.timedep_k10(M=1000)
    obs = np.arange(0, 300, 25)
    before = _gpu.timedep(c, w, TC, obs=obs)[0]
    pm.pm_set_wait_limit(c, 0)
    with pytest.raises(pm.PMError) as e:
        _gpu.timedep(c, w, TC, obs=obs)
    assert e.value.code == pm.PM_ETIMEOUT
    for _ in range(3):  # the setting lasted one call; every CTA freed its tensor memory
        np.testing.assert_array_equal(_gpu.timedep(c, w, TC, obs=obs)[0], before)


def test_persistent_dirichlet_kernel_gives_up_and_the_context_stays_usable(c):
    w = zero_drift_workload(M=512)
    before = _gpu.dirichlet(c, w, TC)
    pm.pm_set_wait_limit(c, 0)
    with pytest.raises(pm.PMError) as e:
        _gpu.dirichlet(c, w, TC)
    assert e.value.code == pm.PM_ETIMEOUT
    after = _gpu.dirichlet(c, w, TC)
    assert after["rc"] == 0
    np.testing.assert_array_equal(after["mean"], before["mean"])


def test_gemm_gives_up_and_the_context_stays_usable(c):
    M, N, K = 256, 128, 512  # eight k-steps: more than the pipeline's stages
    rng = np.random.default_rng(3)
    A = torch.from_numpy(rng.standard_normal((M, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    B = torch.from_numpy(rng.standard_normal((N, K)).astype(np.float32)).to(torch.bfloat16).cuda()
    C0 = torch.empty((M, N), dtype=torch.float32, device="cuda")
    pm.pm_gemm_bf16(c, A, K, B, K, M, N, K, C0, N)
    pm.pm_set_wait_limit(c, 0)
    C1 = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_gemm_bf16(c, A, K, B, K, M, N, K, C1, N)
    assert e.value.code == pm.PM_ETIMEOUT
    assert float(C1.abs().max()) == 0.0  # the epilogue did not run
    C2 = torch.empty_like(C0)
    pm.pm_gemm_bf16(c, A, K, B, K, M, N, K, C2, N)
    assert torch.equal(C2, C0)

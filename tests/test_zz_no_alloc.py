"""pm_forward_timedep_noalloc: the time-dependent map for callers that cannot
allocate device memory (another allocator owns the device, cudaMalloc's
implicit synchronisation is not allowed on their path, or their host forbids
allocation after start-up).  It must give the same results as
pm_forward_timedep on device arrays, call after call, although all calls share
one fixed scratch array, and it must not allocate device memory once the
library's kernels are loaded.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs

torch = pytest.importorskip("torch")
pm = pytest.importorskip("paper_1808_10580_gb300")

pytestmark = pytest.mark.gpu


def _inputs(w, obs, M):
    x = torch.from_numpy(np.ascontiguousarray(w.x[obs])).cuda()
    t = torch.from_numpy(np.ascontiguousarray(w.t[obs])).cuda()
    return x, t, pm.Field(w.K, w.u), pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)


def _with_context(w, obs, M, flags):
    x, t, fld, th = _inputs(w, obs, M)
    mean = torch.empty(len(obs), dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    ctx = pm.pm_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, len(obs), M, w.dt, w.seed, flags, mean, var)
        torch.cuda.synchronize()
    finally:
        pm.pm_destroy(ctx)
    return mean.cpu().numpy(), var.cpu().numpy()


def _without_allocation(w, obs, M, flags):
    x, t, fld, th = _inputs(w, obs, M)
    mean = torch.full((len(obs),), np.nan, dtype=torch.float64, device="cuda")
    var = torch.full_like(mean, np.nan)
    torch.cuda.synchronize()
    pm.pm_forward_timedep_noalloc(fld, w.kappa, th, x, t, len(obs), M, w.dt, w.seed, flags, mean, var,
                                  stream=torch.cuda.current_stream().cuda_stream or None)
    torch.cuda.synchronize()
    return mean.cpu().numpy(), var.cpu().numpy()


def test_matches_the_allocating_entry_point_on_consecutive_calls():
    # Two calls in a row with different shapes and precisions: the shared scratch
    # keeps the first call's contents, which the second call must not depend on.
    cases = [
        (inputs.timedep_k10(M=3000), np.arange(0, 300, 3), 3000, pm.PM_FP32),   # 100 obs, ragged last CTA
        (inputs.plain_fp64_k2(), np.arange(9), 1000, pm.PM_FP64),
    ]
    for w, obs, M, flags in cases:
        ref_mean, ref_var = _with_context(w, obs, M, flags)
        got_mean, got_var = _without_allocation(w, obs, M, flags)
        # same kernels and the same fixed-order reductions: identical up to 1e-12
        np.testing.assert_allclose(got_mean, ref_mean, rtol=0, atol=1e-12)
        np.testing.assert_allclose(got_var, ref_var, rtol=1e-12, atol=1e-12)


def test_rejects_problems_beyond_the_fixed_scratch():
    w = inputs.timedep_k10()
    obs = np.arange(300)
    x, t, fld, th = _inputs(w, obs, 10**6)
    mean = torch.empty(300, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PMError, match="scratch"):
        pm.pm_forward_timedep_noalloc(fld, w.kappa, th, x, t, 300, 10**6, w.dt, w.seed, pm.PM_FP32, mean)


def test_second_call_allocates_no_device_memory():
    # The first call on a device may load the library's kernels (CUDA's lazy
    # module loading); after it, a call of the same shape must leave both the
    # driver's free-memory count and torch's caching allocator unchanged.
    w = inputs.timedep_k10(M=2000)
    obs = np.arange(0, 300, 5)
    x, t, fld, th = _inputs(w, obs, 2000)
    mean = torch.empty(len(obs), dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    stream = torch.cuda.current_stream().cuda_stream or None
    pm.pm_forward_timedep_noalloc(fld, w.kappa, th, x, t, len(obs), 2000, w.dt, w.seed, pm.PM_FP32, mean, var,
                                  stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    first = mean.cpu().numpy()
    pm.pm_forward_timedep_noalloc(fld, w.kappa, th, x, t, len(obs), 2000, w.dt, w.seed, pm.PM_FP32, mean, var,
                                  stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved0
    assert free1 == free0
    np.testing.assert_array_equal(mean.cpu().numpy(), first)


def test_rejects_host_arrays_before_any_work():
    # Host arrays (here numpy) are not device memory of the current device:
    # PM_EINVAL, and the output is left untouched.
    w = inputs.plain_fp64_k2()
    fld, th = pm.Field(w.K, w.u), pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    xh = np.ascontiguousarray(w.x)
    th_ = np.ascontiguousarray(w.t)
    mean = torch.full((len(w.t),), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PMError, match="device pointers"):
        pm.pm_forward_timedep_noalloc(fld, w.kappa, th, xh, th_, len(w.t), 100, w.dt, w.seed, pm.PM_FP64, mean)
    meanh = np.zeros(len(w.t))
    x = torch.from_numpy(xh).cuda()
    t = torch.from_numpy(th_).cuda()
    with pytest.raises(pm.PMError, match="device pointers"):
        pm.pm_forward_timedep_noalloc(fld, w.kappa, th, x, t, len(w.t), 100, w.dt, w.seed, pm.PM_FP64, meanh)
    torch.cuda.synchronize()
    assert bool((mean == 7.0).all())

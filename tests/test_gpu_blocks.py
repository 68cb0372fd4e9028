"""GPU parity of the building blocks of the particle step against the oracle:
Philox words (bit-exact), Box-Muller normals, and the velocity field."""
import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def test_philox_bit_exact_on_a_million_counters(c, orc):
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, size=(1_000_000, 4), dtype=np.uint64).astype(np.uint32)
    key = (0xDEADBEEF, 0x01234567)
    out = np.empty_like(ctr)
    pm.pm_philox(c, ctr, key[0], key[1], len(ctr), out)
    ref = orc.philox(ctr, key)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp32_tensor"])
def test_normals_match_oracle(c, orc, form):
    # fp32: the FP32-pipe kernels' scalar form (sincospif for the angle);
    # fp32_tensor: the tensor-core kernels' packed form (both steps of a Philox
    # block at once, the angle's sin and cos from the library's own series).
    seed = (12345 << 32) | 678
    out = np.empty((4096, 2))
    flags = {"fp64": pm.PM_FP64, "fp32": pm.PM_FP32, "fp32_tensor": pm.PM_FP32 | pm.PM_TENSOR}[form]
    pm.pm_normals(c, seed, 3, 7, 11, 5, 4096, out, flags)
    ref = orc.normals(seed, 3, 7, 11, 5, 4096)
    # float: log and sqrt within a few ulp; sincospif within 1 ulp, the series
    # within 1e-7 absolute
    tol = 1e-13 if form == "fp64" else 4e-6
    print("normals,", form, "largest |GPU - oracle|", np.abs(out - ref).max())
    assert np.abs(out - ref).max() < tol


def test_packed_normals_differ_from_the_scalar_form_by_the_angle_rounding_only(c):
    seed = (777 << 32) | 9
    a, b = np.empty((4096, 2)), np.empty((4096, 2))
    pm.pm_normals(c, seed, 1, 2, 3, 0, 4096, a, pm.PM_FP32)
    pm.pm_normals(c, seed, 1, 2, 3, 0, 4096, b, pm.PM_FP32 | pm.PM_TENSOR)
    rho = np.hypot(a[:, 0], a[:, 1])
    d = np.abs(a - b).max(axis=1)
    # the radius is the same computation in both; the angle's sin and cos differ
    # by at most 1.2e-7 (1 ulp of sincospif plus the series' 8.4e-8)
    print("packed vs scalar float normals: identical", np.mean(d == 0), "largest difference / radius",
          (d / rho).max())
    assert np.all(d <= rho * 1.5e-7 + 1e-12)


@pytest.mark.parametrize("K", [0, 1, 2, 3, 4, 5, 6, 8, 10, 12, 16])
@pytest.mark.parametrize("fp64", [False, True])
def test_velocity_matches_direct_sum(c, orc, K, fp64):
    u = inputs.prior_field(K, 100 + K)
    rng = np.random.default_rng(K)
    x = np.concatenate([rng.random((4000, 2)), rng.random((1000, 2)) * 2 - 0.5])  # also outside [0,1)^2
    v = np.empty_like(x)
    pm.pm_velocity(c, pm.Field(K, u), x, len(x), v, pm.PM_FP64 if fp64 else pm.PM_FP32)
    ref = orc.velocity(K, u, x)
    modes = orc.half_modes(K).astype(float)
    # bound on the size of the terms of the sum: sum_h 2 pi |k_h| (|a_h| + |b_h|)
    scale = float((2 * np.pi * np.sqrt((modes ** 2).sum(1)) * np.abs(u.reshape(-1, 2)).sum(1)).sum()) if K else 1.0
    tol = (1e-13 if fp64 else 2e-6 * max(K, 1)) * scale
    assert np.abs(v - ref).max() <= tol, (np.abs(v - ref).max(), tol)


def test_own_sincos_of_two_pi_x_meets_its_error_bound():
    # The tensor-core kernels' sin/cos of 2 pi x (quarter-turn reduction, Taylor
    # series in turns) against float64 on 2e6 random points of [0, 1), a dense
    # grid, the quarter turns and points around them, and positions a little
    # outside [0, 1): absolute error below 1e-7, relative below 2 ulp where
    # |value| > 1e-6 (near the exact zeros the float64 reference itself is
    # rounded at 1e-16 while the float result is exact or tiny).
    c = _gpu.ctx()
    try:
        rng = np.random.default_rng(42)
        q = np.float32([0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 1.0])
        x = np.concatenate([rng.random(2_000_000).astype(np.float32), np.linspace(0, 1, 100_001, dtype=np.float32),
                            q, np.nextafter(q, np.float32(2)), np.nextafter(q, np.float32(-2)),
                            np.float32([-0.3, -1e-3, 1.2, 2.7])])
        xt = torch.from_numpy(x).cuda()
        s = torch.empty_like(xt)
        co = torch.empty_like(xt)
        pm.pm_sincos_turns(c, xt, s, co)
        s, co = s.cpu().numpy().astype(np.float64), co.cpu().numpy().astype(np.float64)
        ts, tc = np.sin(2 * np.pi * x.astype(np.float64)), np.cos(2 * np.pi * x.astype(np.float64))
        assert np.abs(s - ts).max() < 1e-7 and np.abs(co - tc).max() < 1e-7
        for got, ref in ((s, ts), (co, tc)):
            big = np.abs(ref) > 1e-6
            ulp = np.spacing(np.abs(ref[big]).astype(np.float32)).astype(np.float64)
            assert (np.abs(got[big] - ref[big]) / ulp).max() < 2.0
    finally:
        pm.pm_destroy(c)

"""The float pre-test of the disk kernels' exit decision (`exits_disk`, used by
the tensor-core disk and batched maps for Algorithm 2's first-exit test).

A float path's position is compensated, X = hi + lo with |lo| <= ulp(hi)/2.
The kernels first compare the float value q = hi1^2 + hi2^2 (one rounded
product and one fused multiply-add) with R2hi = float(R^2) and run the exact
compensated test only when |q - R2hi| <= 2^-16 R2hi.  That is sound when the
float value's error near the circle stays well below the band: it is at most
2^-21 R^2 there.  This emulates the float arithmetic exactly in numpy (a
float32 rounding of a float64 value that holds the exact product) and checks,
on points within a few band widths of circles of several radii, that outside
the band the float decision equals the sign of |X|^2 - R^2, and that the error
bound holds."""
import numpy as np


def _f32(v):
    return np.asarray(v, dtype=np.float64).astype(np.float32)


def _float_excess(xh, yh, R2hi):
    # p2 = fl(y^2); q = fma(x, x, p2): the product x*x is exact in float64
    p2 = _f32(yh.astype(np.float64) * yh)
    q = _f32(xh.astype(np.float64) * xh + p2.astype(np.float64))
    return q, (q - R2hi).astype(np.float32)


def test_float_exit_test_outside_the_band_has_the_exact_sign():
    rng = np.random.default_rng(5)
    n = 200_000
    for R in (1.0, 0.7, 3.0):
        R2 = R * R
        R2hi = np.float32(R2)
        band = np.float32(np.ldexp(np.float64(R2hi), -16))
        # half within a few band widths, half within a few float spacings of R
        r = R * (1.0 + np.concatenate([rng.uniform(-4e-5, 4e-5, n // 2), rng.uniform(-4e-7, 4e-7, n // 2)]))
        phi = rng.uniform(0.0, 2.0 * np.pi, n)
        x, y = r * np.cos(phi), r * np.sin(phi)
        xh, yh = _f32(x), _f32(y)
        xl, yl = _f32(x - xh), _f32(y - yh)  # the compensated parts
        X = xh.astype(np.float64) + xl
        Y = yh.astype(np.float64) + yl
        exact = X * X + Y * Y - R2
        q, d = _float_excess(xh, yh, R2hi)
        outside = np.abs(d) > band
        assert outside.sum() > n // 4 and (~outside).sum() > 1000
        assert np.array_equal(d[outside] > 0, exact[outside] > 0)
        err = np.abs(q.astype(np.float64) - (X * X + Y * Y))
        assert err.max() <= np.ldexp(R2, -21), err.max() / R2


def test_points_far_from_the_circle_never_need_the_exact_test():
    # a path well inside or outside decides in float: the band is a few
    # millionths of R^2 wide
    rng = np.random.default_rng(6)
    R2hi = np.float32(1.0)
    band = np.float32(np.ldexp(1.0, -16))
    r = np.concatenate([rng.uniform(0.0, 0.999, 10_000), rng.uniform(1.001, 2.0, 10_000)])
    phi = rng.uniform(0.0, 2.0 * np.pi, r.size)
    _, d = _float_excess(_f32(r * np.cos(phi)), _f32(r * np.sin(phi)), R2hi)
    assert np.all(np.abs(d) > band)
    assert np.array_equal(d > 0, r > 1.0)

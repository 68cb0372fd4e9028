"""Why the time-dependent tensor-core kernels may wrap positions into [0, 1)
only every 32nd step: their sin and cos of 2 pi x (sincos_turns2) first reduce x
to r = x - q/4 with q = rint(4x) (by adding and subtracting 1.5 2^23, then one
FMA), and everything after depends only on r and on q mod 4.  For a float
position X in [1, 2) and the wrapped X - 1 (exact in float), this emulates
those float steps exactly in numpy and checks that r is the same bits and q
differs by 4, so the harmonics of X and X - 1 are the same bits.  For X in
[-1, 0), X + 1 is a float only for part of the values: the wrap's two-sum keeps
the rest in the position's low word (under either schedule), and wherever the
shift is exact the same holds."""
import numpy as np

ROUND = np.float32(1.5 * 2 ** 23)


def _reduce(x):
    x = np.asarray(x, dtype=np.float32)
    # t = fma(x, 4, 1.5 2^23): 4x is exact, one rounding to float
    t = (x.astype(np.float64) * 4.0 + np.float64(ROUND)).astype(np.float32)
    q = (t - ROUND).astype(np.float32)  # exact
    # r = fma(q, -0.25, x): one rounding of the exact value
    r = (q.astype(np.float64) * -0.25 + x.astype(np.float64)).astype(np.float32)
    return q, r


def test_reduced_argument_and_quadrant_repeat_with_period_one():
    rng = np.random.default_rng(11)
    n = 1_000_000
    for lo, hi, shift in ((1.0, 2.0, -1.0), (-1.0, 0.0, 1.0)):
        X = rng.uniform(lo, hi, n).astype(np.float32)
        W = (X + np.float32(shift)).astype(np.float32)
        exact = W.astype(np.float64) == X.astype(np.float64) + shift
        if shift < 0:
            assert exact.all()  # Sterbenz: X - 1 is a float for X in [1, 2)
        else:
            # the rounding of X + 1, which the wrap keeps in the low word, is at most
            # half a float spacing of the result
            gap = np.abs(W.astype(np.float64) - (X.astype(np.float64) + shift))
            assert np.all(gap <= np.spacing(W).astype(np.float64) / 2)
            assert exact.sum() > n // 20
            X, W = X[exact], W[exact]
        n_ok = X.size
        qX, rX = _reduce(X)
        qW, rW = _reduce(W)
        assert np.array_equal(rX.view(np.uint32), rW.view(np.uint32))
        assert np.array_equal(qX.astype(np.float64) - qW.astype(np.float64), np.full(n_ok, -4.0 * shift))
        # the reduction is exact: x - q/4 in [-1/8, 1/8]
        assert np.array_equal(rX.astype(np.float64), X.astype(np.float64) - qX.astype(np.float64) / 4)
        assert np.abs(rX).max() <= 0.125


def test_quadrant_boundaries():
    # the quarter-turn points themselves and their float neighbours
    k = np.arange(-8, 9, dtype=np.float64) / 4.0
    X = np.concatenate([k, np.nextafter(k.astype(np.float32), np.float32(np.inf)),
                        np.nextafter(k.astype(np.float32), np.float32(-np.inf))]).astype(np.float32)
    X = X[(X >= 1.0) & (X < 2.0)]
    qX, rX = _reduce(X)
    qW, rW = _reduce((X - np.float32(1.0)).astype(np.float32))
    assert np.array_equal(rX.view(np.uint32), rW.view(np.uint32))
    assert np.all(qX - qW == 4)

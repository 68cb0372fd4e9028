"""Pins of the oracle's random-number layer: Philox4x32-10 against the published
known-answer vectors, the Box-Muller normals against the normal law."""
import os

import numpy as np
import pytest
from scipy import stats

from tests import _bruteforce as bf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(orc, ctr, key, want):
    got = orc.philox([ctr], key)[0]
    assert [int(v) for v in got] == want
    assert bf.philox(ctr, key) == want


def test_philox_batch_matches_scalar_restatement(orc):
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x12345678, 0x9abcdef0]
    got = orc.philox(ctr, key)
    for c, g in zip(ctr, got):
        assert bf.philox(c, key) == [int(v) for v in g]


def test_normals_follow_counter_layout(orc):
    seed = (7 << 32) | 99
    xi = orc.normals(seed, 3, 5, 11, 0, 6)
    for n in range(6):
        ref = bf.normals(seed, 3, 5, 11, n)
        assert np.allclose(xi[n], ref, rtol=0, atol=1e-15)


def test_normals_are_standard_normal(orc):
    # 2 x 100,000 draws from distinct paths: KS against N(0,1), moments, independence.
    xi = np.concatenate([orc.normals(2024, 0, j, 0, 0, 1000) for j in range(100)])
    for c in range(2):
        z = xi[:, c]
        assert stats.kstest(z, "norm").pvalue > 1e-3
        assert abs(z.mean()) < 5 / np.sqrt(len(z))
        assert abs(z.var() - 1) < 5 * np.sqrt(2 / len(z))
    assert abs(np.corrcoef(xi[:, 0], xi[:, 1])[0, 1]) < 5 / np.sqrt(len(xi))
    # neighbouring steps are uncorrelated too
    assert abs(np.corrcoef(xi[:-1, 0], xi[1:, 0])[0, 1]) < 5 / np.sqrt(len(xi))


def test_uniforms_never_reach_zero_or_one(orc):
    # The extreme words give the extreme uniforms 2^-24 and 1 - 2^-24, so log() is finite.
    assert ((0 >> 9) * 2 + 1) / 2 ** 24 == 2.0 ** -24
    assert (((2 ** 32 - 1) >> 9) * 2 + 1) / 2 ** 24 == 1 - 2.0 ** -24

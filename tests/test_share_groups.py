"""Host logic of shared paths (PM_SHARE_PATHS), no GPU: the groups the library
forms match their definition (observations at bit-identical points, the RNG
stream of the lowest member index, one path per group running to the group's
largest step count), written out here with plain Python loops."""
import math

import numpy as np
import pytest

import paper_1808_10580_gb300 as pm
from paper_1808_10580_gb300 import inputs


def groups_by_definition(x, t, dt):
    N = [0 if tj == 0 else math.ceil(tj / dt - 1e-9) for tj in t]
    by_point = {}
    for j in range(len(t)):
        by_point.setdefault((x[j, 0].tobytes(), x[j, 1].tobytes()), []).append(j)
    groups = [(max(N[j] for j in js), min(js), js) for js in by_point.values()]
    groups.sort(key=lambda g: (-g[0], g[1]))          # launch order: longest first, then stream
    group_of, stream_of = np.empty(len(t), np.int32), np.empty(len(t), np.int32)
    for gi, (nmax, s, js) in enumerate(groups):
        for j in js:
            group_of[j], stream_of[j] = gi, s
    return group_of, stream_of, len(groups), sum(g[0] for g in groups)


def test_headline_workload_groups():
    w = inputs.timedep_k10()
    gof, sof, ng, sp = pm.pm_path_groups(w.x, w.t, w.dt)
    # 100 points x t in {0.25, 0.5, 1}: 100 groups, 1000 steps per path index
    # instead of 1750 per observation triple
    assert ng == 100 and sp == 100 * 1000
    assert np.array_equal(sof[:100], np.arange(100)) and np.array_equal(sof[200:], np.arange(100))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_layouts_match_definition(seed):
    rng = np.random.default_rng(seed)
    pts = rng.random((7, 2))
    n = 40
    x = pts[rng.integers(0, 7, n)].copy()
    x[5] = np.nextafter(x[5], 2.0)                    # one point a single ulp away: its own group
    t = rng.choice([0.0, 0.1, 0.25, 0.2501, 0.7, 1.0], n)
    dt = 0.003
    got = pm.pm_path_groups(x, t, dt)
    want = groups_by_definition(x, t, dt)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert got[2:] == want[2:]


def test_no_shared_points_is_one_group_per_observation():
    x = np.random.default_rng(3).random((9, 2))
    t = np.linspace(0.1, 0.9, 9)
    gof, sof, ng, sp = pm.pm_path_groups(x, t, 0.01)
    assert ng == 9 and np.array_equal(sof, np.arange(9))
    assert sp == sum(math.ceil(tt / 0.01 - 1e-9) for tt in t)


def test_invalid_times_are_rejected():
    x = np.zeros((2, 2))
    for bad in ([0.1, -1.0], [0.1, np.nan]):
        with pytest.raises(pm.PMError):
            pm.pm_path_groups(x, np.array(bad), 0.01)

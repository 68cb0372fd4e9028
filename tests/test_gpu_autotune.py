"""The autotuner of the persistent launches: it picks a CTAs-per-SM count in
[1, occupancy limit] and, for the tensor-core kernels, the number of step
pairs between lane refills; neither changes the results, the cache file
round-trips both, and PM_AUTOTUNE=0 restores the occupancy limit."""
import os

import numpy as np
import pytest

from paper_1808_10580_gb300 import inputs
from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm
torch = _gpu.torch
TC = pm.PM_FP32 | pm.PM_TENSOR


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def batch_problem():
    from tests.test_gpu_batched import small_instances
    return small_instances(B=8, M=4096)


def test_batched_autotune_changes_the_grid_not_the_results():
    c = _gpu.ctx()
    try:
        ws = batch_problem()
        rc, m0, v0, _ = _gpu.batched(c, ws, flags=TC)
        resident = pm.pm_last_grid(c) // sms()
        b, _ = _gpu.batch_from_workloads(ws, device=True)
        best = pm.pm_autotune_batched(c, b, TC)
        assert 1 <= best <= resident
        rc, m1, v1, _ = _gpu.batched(c, ws, flags=TC)
        assert pm.pm_last_grid(c) == best * sms()
        assert np.array_equal(m0, m1) and np.array_equal(v0, v1)
        pm.pm_set_ctas_per_sm(c, pm.PM_TUNE_BATCHED, 10, pm.PM_TENSOR, 1)
        rc, m2, _, _ = _gpu.batched(c, ws, flags=TC)
        assert pm.pm_last_grid(c) == sms() and np.array_equal(m0, m2)
        os.environ["PM_AUTOTUNE"] = "0"
        try:
            _gpu.batched(c, ws, flags=TC)
            assert pm.pm_last_grid(c) == resident * sms()
        finally:
            del os.environ["PM_AUTOTUNE"]
    finally:
        pm.pm_destroy(c)


def test_dirichlet_autotune_changes_the_grid_not_the_results():
    c = _gpu.ctx()
    try:
        w = inputs.dirichlet_disk_k10(M=4096)
        w.max_steps = 4000
        r0 = _gpu.dirichlet(c, w, TC)
        best = pm.pm_autotune_dirichlet(c, pm.Field(w.K, w.u), w.drift_scale, w.kappa,
                                        pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b), w.x, len(w.x),
                                        w.M, w.dt, w.max_steps, w.seed, TC)
        r1 = _gpu.dirichlet(c, w, TC)
        assert pm.pm_last_grid(c) == best * sms()
        assert np.array_equal(r0["mean"], r1["mean"]) and np.array_equal(r0["var"], r1["var"])
    finally:
        pm.pm_destroy(c)


def test_dirichlet_autotune_at_a_wide_bound():
    # K = 24 on the tensor cores: the tuner's candidates, then the same results
    c = _gpu.ctx()
    try:
        w = inputs.dirichlet_disk_k10(M=4096)
        w.K, w.u = 24, inputs.prior_field(24, 624)
        w.max_steps = 2000
        r0 = _gpu.dirichlet(c, w, TC)
        resident = pm.pm_last_grid(c) // sms()
        best = pm.pm_autotune_dirichlet(c, pm.Field(w.K, w.u), w.drift_scale, w.kappa,
                                        pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b), w.x, len(w.x),
                                        w.M, w.dt, w.max_steps, w.seed, TC)
        assert 1 <= best <= resident
        r1 = _gpu.dirichlet(c, w, TC)
        assert pm.pm_last_grid(c) == best * sms()
        assert np.array_equal(r0["mean"], r1["mean"]) and np.array_equal(r0["var"], r1["var"])
    finally:
        pm.pm_destroy(c)


def test_cache_file_round_trip(tmp_path):
    path = tmp_path / "tune.json"
    os.environ["PM_AUTOTUNE_CACHE"] = str(path)
    try:
        c = _gpu.ctx()
        ws = batch_problem()
        b, _ = _gpu.batch_from_workloads(ws, device=True)
        best = pm.pm_autotune_batched(c, b, TC)
        pm.pm_destroy(c)
        text = path.read_text()
        name = torch.cuda.get_device_properties(0).name
        assert f'"{name}|{pm.PM_TUNE_BATCHED}|10|{pm.PM_TENSOR}": {best}' in text
        c2 = _gpu.ctx()                       # a new context reads the choice
        _gpu.batched(c2, ws, flags=TC)
        assert pm.pm_last_grid(c2) == best * sms()
        pm.pm_destroy(c2)
    finally:
        del os.environ["PM_AUTOTUNE_CACHE"]


@pytest.mark.parametrize("kind", ["dirichlet", "batched"])
def test_refill_interval_changes_nothing_in_the_results(kind):
    # Every path's random numbers are keyed by its own step index: how often
    # the lanes refill is a launch shape, not part of the arithmetic.
    c = _gpu.ctx()
    try:
        if kind == "dirichlet":
            w = inputs.dirichlet_disk_k10(M=2048)
            w.max_steps = 3000
            run = lambda: _gpu.dirichlet(c, w, TC, want_paths=True)
            key = pm.PM_TUNE_DIRICHLET
        else:
            ws = batch_problem()
            run = lambda: _gpu.batched(c, ws, flags=TC)
            key = pm.PM_TUNE_BATCHED
        ref = run()
        for pairs in (1, 2, 8, 16):
            pm.pm_set_refill_pairs(c, key, 10, pm.PM_TENSOR, pairs)
            assert pm.pm_tuned_shape(c, key, 10, pm.PM_TENSOR)[1] == pairs
            got = run()
            if kind == "dirichlet":
                assert np.array_equal(got["g"], ref["g"]) and np.array_equal(got["steps"], ref["steps"])
                assert np.array_equal(got["mean"], ref["mean"])
            else:
                assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    finally:
        pm.pm_destroy(c)


def test_autotuner_records_both_shapes_and_the_cache_keeps_them(tmp_path):
    path = tmp_path / "tune2.json"
    os.environ["PM_AUTOTUNE_CACHE"] = str(path)
    try:
        c = _gpu.ctx()
        ws = batch_problem()
        b, _ = _gpu.batch_from_workloads(ws, device=True)
        best = pm.pm_autotune_batched(c, b, TC)
        ctas, pairs = pm.pm_tuned_shape(c, pm.PM_TUNE_BATCHED, 10, pm.PM_TENSOR)
        assert ctas == best and pairs in (1, 2, 4, 8, 16)
        pm.pm_destroy(c)
        name = torch.cuda.get_device_properties(0).name
        assert f'"{name}|{pm.PM_TUNE_BATCHED}|10|{pm.PM_TENSOR}|refill": {pairs}' in path.read_text()
        c2 = _gpu.ctx()
        assert pm.pm_tuned_shape(c2, pm.PM_TUNE_BATCHED, 10, pm.PM_TENSOR) == (ctas, pairs)
        pm.pm_destroy(c2)
    finally:
        del os.environ["PM_AUTOTUNE_CACHE"]

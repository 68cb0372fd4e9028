"""FP64 CPU oracle for the particle forward maps (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it.

The C part (``pm_oracle.c``) holds Philox4x32-10, Box-Muller, the direct-sum
velocity and the path loops of Algorithms 1 and 2.  This wrapper adds the
estimator (plain numpy mean and unbiased variance, Algorithm 1/2's final
averaging step) and loads the library built by ``oracle/build.py``.
The MLP and MCMC parts of the oracle live in ``oracle/mlp.py`` and
``oracle/mcmc.py``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.library_path()
        if not os.path.exists(path) or _build.stale():
            _build.build()
        L = C.CDLL(path)
        d = C.POINTER(C.c_double)
        i32 = C.POINTER(C.c_int32)
        i64 = C.POINTER(C.c_int64)
        u32 = C.POINTER(C.c_uint32)
        L.or_philox4x32_10.argtypes = [u32, u32, u32]
        L.or_philox_batch.argtypes = [u32, u32, u32, C.c_int64]
        L.or_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, C.c_int64, d]
        L.or_num_half_modes.argtypes = [C.c_int32]
        L.or_num_half_modes.restype = C.c_int64
        L.or_half_modes.argtypes = [C.c_int32, i32]
        L.or_count_disk_modes.argtypes = [C.c_double]
        L.or_count_disk_modes.restype = C.c_int64
        L.or_velocity.argtypes = [C.c_int32, d, C.c_int64, d, d]
        L.or_stream_function.argtypes = [C.c_int32, d, C.c_int64, d, d]
        L.or_theta0.argtypes = [C.c_int32, i32, d, d, C.c_int64, d, d]
        L.or_num_steps.argtypes = [C.c_double, C.c_double]
        L.or_num_steps.restype = C.c_int64
        L.or_timedep_paths.argtypes = [C.c_int32, d, C.c_double, C.c_int32, i32, d, d, d, d,
                                       C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_uint64,
                                       C.c_uint32, i64, C.c_int32, d, d]
        L.or_timedep_paths.restype = C.c_int32
        L.or_dirichlet_paths.argtypes = [C.c_int32, d, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int32, d, d, d, C.c_int64, C.c_int64,
                                         C.c_int64, C.c_double, C.c_int64, C.c_uint64, C.c_uint32,
                                         i64, C.c_int32, d, i64, d]
        L.or_dirichlet_paths.restype = C.c_int32
        L.or_dirichlet_general_paths.argtypes = [C.c_int32, d, C.c_double, d, d, C.c_int32, C.c_double,
                                                 C.c_double, C.c_double, C.c_int32, d, d, C.c_int32, C.c_double,
                                                 d, d, d, C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_int64,
                                                 C.c_uint64, C.c_uint32, i64, C.c_int32, d, i64, d]
        L.or_dirichlet_general_paths.restype = C.c_int32
        L.or_square_bvp_paths.argtypes = [d, C.c_double, C.c_int32, d, C.c_double, C.c_double, C.c_double, d,
                                          C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_int64, C.c_uint64,
                                          C.c_uint32, i64, C.c_int32, d, i64]
        L.or_square_bvp_paths.restype = C.c_int32
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox(ctr, key):
    """Philox4x32-10 of counters ``ctr`` [n, 4] under ``key`` [2] -> [n, 4] uint32."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().or_philox_batch(_p(ctr, C.c_uint32), _p(key, C.c_uint32), _p(out, C.c_uint32), ctr.shape[0])
    return out


def normals(seed, b, j, i, n0, count):
    """Normals (xi1, xi2) of steps n0..n0+count-1 of path (b, j, i) -> [count, 2]."""
    out = np.empty((count, 2))
    lib().or_normals(seed, b, j, i, n0, count, _p(out, C.c_double))
    return out


def half_modes(K):
    H = lib().or_num_half_modes(K)
    out = np.empty((H, 2), dtype=np.int32)
    if H:
        lib().or_half_modes(K, _p(out, C.c_int32))
    return out


def count_disk_modes(r):
    return int(lib().or_count_disk_modes(float(r)))


def velocity(K, u, x):
    x = _f64(x).reshape(-1, 2)
    u = _f64(u)
    v = np.empty_like(x)
    lib().or_velocity(K, _p(u, C.c_double), x.shape[0], _p(x, C.c_double), _p(v, C.c_double))
    return v


def stream_function(K, u, x):
    x = _f64(x).reshape(-1, 2)
    u = _f64(u)
    out = np.empty(x.shape[0])
    lib().or_stream_function(K, _p(u, C.c_double), x.shape[0], _p(x, C.c_double), _p(out, C.c_double))
    return out


def theta0(th, x):
    x = _f64(x).reshape(-1, 2)
    k = np.ascontiguousarray(th.k, dtype=np.int32)
    a, b = _f64(th.a), _f64(th.b)
    out = np.empty(x.shape[0])
    lib().or_theta0(len(a), _p(k, C.c_int32), _p(a, C.c_double), _p(b, C.c_double), x.shape[0],
                    _p(x, C.c_double), _p(out, C.c_double))
    return out


def num_steps(t, dt):
    return int(lib().or_num_steps(float(t), float(dt)))


def _ids(obs_id, n):
    if obs_id is None:
        return None
    ids = np.ascontiguousarray(np.asarray(obs_id, dtype=np.int64).reshape(-1))
    assert ids.shape[0] == n
    return ids


def timedep_paths(K, u, kappa, th, x, t, dt, seed, i0=0, npaths=1, inst=0, nthreads=0,
                  want_x=False, obs_id=None):
    """Per-path g of Algorithm 1 -> g [n_obs, npaths] (and end points [n_obs, npaths, 2]).

    ``obs_id`` gives the observation index j the RNG counter uses for each row
    of ``x`` (default: the row number)."""
    x = _f64(x).reshape(-1, 2)
    t = _f64(t).reshape(-1)
    u = _f64(u)
    k = np.ascontiguousarray(th.k, dtype=np.int32).reshape(-1, 2)
    a, b = _f64(th.a), _f64(th.b)
    n_obs = x.shape[0]
    g = np.empty((n_obs, npaths))
    xe = np.empty((n_obs, npaths, 2)) if want_x else None
    ids = _ids(obs_id, n_obs)
    nt = lib().or_timedep_paths(K, _p(u, C.c_double), kappa, len(a), _p(k, C.c_int32),
                                _p(a, C.c_double), _p(b, C.c_double), _p(x, C.c_double),
                                _p(t, C.c_double), n_obs, i0, npaths, dt, seed, inst,
                                _p(ids, C.c_int64) if ids is not None else None, nthreads,
                                _p(g, C.c_double),
                                _p(xe, C.c_double) if want_x else None)
    if nt < 0:
        raise MemoryError("oracle allocation failed")
    return (g, xe) if want_x else g


def dirichlet_paths(K, u, drift_scale, kappa, gd, x, dt, max_steps, seed, i0=0, npaths=1, inst=0,
                    nthreads=0, want_x=False, obs_id=None):
    """Per-path g and exit step of Algorithm 2 -> (g [n_obs, npaths], steps [n_obs, npaths])."""
    x = _f64(x).reshape(-1, 2)
    u = _f64(u)
    ga, gb = _f64(gd.a), _f64(gd.b)
    n_ang = len(ga)
    assert len(gb) == n_ang
    n_obs = x.shape[0]
    g = np.empty((n_obs, npaths))
    st = np.empty((n_obs, npaths), dtype=np.int64)
    xe = np.empty((n_obs, npaths, 2)) if want_x else None
    ids = _ids(obs_id, n_obs)
    nt = lib().or_dirichlet_paths(K, _p(u, C.c_double), drift_scale, kappa, gd.R, gd.quad,
                                  gd.f_const, n_ang, _p(ga, C.c_double), _p(gb, C.c_double),
                                  _p(x, C.c_double), n_obs, i0, npaths, dt, max_steps, seed, inst,
                                  _p(ids, C.c_int64) if ids is not None else None, nthreads, _p(g, C.c_double), _p(st, C.c_int64),
                                  _p(xe, C.c_double) if want_x else None)
    if nt < 0:
        raise MemoryError("oracle allocation failed")
    return (g, st, xe) if want_x else (g, st)


def dirichlet_general_paths(K, u, drift_scale, gen, gd, x, dt, max_steps, seed, i0=0, npaths=1, inst=0,
                            nthreads=0, want_x=False, obs_id=None):
    """Per-path values and exit steps of Algorithm 2 in the disk with the
    general forcing and diagonal affine diffusion of ``gen`` (attributes s0[2],
    s1[2], milstein, n_src sources at c [n_src, 2] with amplitudes F and width
    w) -> (g [n_obs, npaths], steps [n_obs, npaths] (, exit points))."""
    x = _f64(x).reshape(-1, 2)
    u = _f64(u)
    ga, gb = _f64(gd.a), _f64(gd.b)
    c = _f64(gen.c).reshape(-1, 2)
    F = _f64(gen.F).reshape(-1)
    s0, s1 = _f64(gen.s0).reshape(2), _f64(gen.s1).reshape(2)
    n_obs = x.shape[0]
    g = np.empty((n_obs, npaths))
    st = np.empty((n_obs, npaths), dtype=np.int64)
    xe = np.empty((n_obs, npaths, 2)) if want_x else None
    ids = _ids(obs_id, n_obs)
    nt = lib().or_dirichlet_general_paths(K, _p(u, C.c_double), drift_scale, _p(s0, C.c_double), _p(s1, C.c_double),
                                          int(gen.milstein), gd.R, gd.quad, gd.f_const, len(ga), _p(ga, C.c_double),
                                          _p(gb, C.c_double), len(F), float(gen.w), _p(c, C.c_double),
                                          _p(F, C.c_double), _p(x, C.c_double), n_obs, i0, npaths, dt, max_steps,
                                          seed, inst, _p(ids, C.c_int64) if ids is not None else None, nthreads,
                                          _p(g, C.c_double), _p(st, C.c_int64),
                                          _p(xe, C.c_double) if want_x else None)
    if nt < 0:
        raise MemoryError("oracle allocation failed")
    return (g, st, xe) if want_x else (g, st)


def square_bvp_paths(prob, x, dt, max_steps, seed, i0=0, npaths=1, inst=0, nthreads=0, obs_id=None):
    """Per-path values of the optimal-forcing problem in the unit square
    (Section 4, Eq. bvp:ex1, by Algorithm 2 / Theorem 3.2) -> (out [n_obs,
    n_src + 1, npaths]: g(X_tau) then the time integrals of each source
    profile, exit steps [n_obs, npaths])."""
    x = _f64(x).reshape(-1, 2)
    c = _f64(prob.c).reshape(-1, 2)
    b = _f64(prob.b).reshape(2)
    n_obs, n_src = x.shape[0], c.shape[0]
    out = np.empty((n_obs, n_src + 1, npaths))
    st = np.empty((n_obs, npaths), dtype=np.int64)
    ids = _ids(obs_id, n_obs)
    nt = lib().or_square_bvp_paths(_p(b, C.c_double), prob.kappa, n_src, _p(c, C.c_double), prob.w, prob.g_cos,
                                   prob.g_quad, _p(x, C.c_double), n_obs, i0, npaths, dt, max_steps, seed, inst,
                                   _p(ids, C.c_int64) if ids is not None else None, nthreads, _p(out, C.c_double),
                                   _p(st, C.c_int64))
    if nt < 0:
        raise ValueError("oracle: at most 16 sources")
    return out, st


def estimate(g):
    """Algorithm 1/2's final step, per observation: sample mean, unbiased
    variance (n-1) and standard error of the per-path values g [n_obs, M]."""
    g = np.asarray(g, dtype=np.float64)
    M = g.shape[1]
    mean = g.mean(axis=1)
    var = g.var(axis=1, ddof=1) if M > 1 else np.zeros(g.shape[0])
    return mean, var, np.sqrt(var / M)


def timedep_estimate(w, i0=0, npaths=None, obs=None, nthreads=0):
    """Oracle estimate for a TimedepWorkload (optionally a subset of observations/paths)."""
    npaths = w.M if npaths is None else npaths
    obs = np.arange(len(w.t)) if obs is None else np.asarray(obs)
    g = timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, w.seed, i0, npaths,
                      nthreads=nthreads, obs_id=obs)
    return estimate(g), g

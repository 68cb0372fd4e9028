"""ctypes binding of the C ABI in include/pm.h (argument marshalling only).

Every function here has the name of its C entry point and forwards its
arguments unchanged; all arithmetic runs in the CUDA library
``_build/libpm_gb300.so``.  Arrays may be numpy arrays (host pointers) or
CUDA torch tensors (device pointers, which set PM_DEVICE_PTRS).  If the
library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PM_OK = 0
PM_EINVAL = -1
PM_ENOMEM = -2
PM_ECUDA = -3
PM_ETIMEOUT = -4
PM_WARN_UNEXITED = 1

PM_FP32 = 0
PM_FP64 = 1
PM_DEVICE_PTRS = 2
PM_ASYNC = 4
PM_TENSOR = 8
PM_SHARE_PATHS = 16
PM_TUNE_DIRICHLET = 0
PM_TUNE_BATCHED = 1


class PMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pm error {code}: {msg}")
        self.code = code


class pm_field(C.Structure):
    _fields_ = [("K", C.c_int32), ("reserved", C.c_int32), ("u", C.POINTER(C.c_double))]


class pm_fourier(C.Structure):
    _fields_ = [("n", C.c_int32), ("reserved", C.c_int32), ("k", C.POINTER(C.c_int32)),
                ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class pm_dirichlet_data(C.Structure):
    _fields_ = [("R", C.c_double), ("quad", C.c_double), ("f_const", C.c_double), ("n_ang", C.c_int32),
                ("reserved", C.c_int32), ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double))]


class pm_path_opts(C.Structure):
    _fields_ = [("path_offset", C.c_int64), ("instance", C.c_uint32), ("reserved", C.c_int32),
                ("g_out", C.c_void_p), ("x_out", C.c_void_p)]


PM_KIND_TIMEDEP = 0
PM_KIND_DIRICHLET = 1


class pm_instance(C.Structure):
    _fields_ = [("kind", C.c_int32), ("stream", C.c_uint32), ("u", C.c_void_p), ("kappa", C.c_double),
                ("dt", C.c_double), ("drift_scale", C.c_double), ("max_steps", C.c_int64), ("row0", C.c_int64),
                ("n_obs", C.c_int64), ("M", C.c_int64), ("seed", C.c_uint64)]


class pm_batch(C.Structure):
    _fields_ = [("K", C.c_int32), ("B", C.c_int32), ("inst", C.POINTER(pm_instance)),
                ("theta0", C.POINTER(pm_fourier)), ("disk", C.POINTER(pm_dirichlet_data)), ("x", C.c_void_p),
                ("t", C.c_void_p), ("n_rows", C.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads the CUDA library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build.stale()):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run paper_1808_10580_gb300/build.py")
    L = C.CDLL(path)
    vp = C.c_void_p
    i64, u32, i32, dbl = C.c_int64, C.c_uint32, C.c_int32, C.c_double
    L.pm_version.restype = C.c_int
    L.pm_create.argtypes = [C.POINTER(vp), C.c_int, vp]
    L.pm_destroy.argtypes = [vp]
    L.pm_destroy.restype = None
    L.pm_last_error.restype = C.c_char_p
    L.pm_stream.argtypes = [vp]
    L.pm_stream.restype = vp
    L.pm_forward_timedep.argtypes = [vp, C.POINTER(pm_field), dbl, C.POINTER(pm_fourier), vp, vp, i64, i64, dbl,
                                     C.c_uint64, u32, vp, vp, C.POINTER(pm_path_opts)]
    L.pm_forward_dirichlet.argtypes = [vp, C.POINTER(pm_field), dbl, dbl, C.POINTER(pm_dirichlet_data), vp, i64,
                                       i64, dbl, i64, C.c_uint64, u32, vp, vp, vp, vp, C.POINTER(pm_path_opts)]
    L.pm_forward_dirichlet_general.argtypes = [vp, C.POINTER(pm_field), dbl, C.POINTER(pm_dirichlet_data),
                                               C.POINTER(pm_diffusion_forcing), vp, i64, i64, dbl, i64, C.c_uint64,
                                               u32, vp, vp, vp, vp, C.POINTER(pm_path_opts)]
    L.pm_philox.argtypes = [vp, vp, u32, u32, i64, vp, u32]
    L.pm_normals.argtypes = [vp, C.c_uint64, u32, u32, u32, i64, i64, vp, u32]
    L.pm_velocity.argtypes = [vp, C.POINTER(pm_field), vp, i64, vp, u32]
    L.pm_forward_timedep_noalloc.argtypes = [C.POINTER(pm_field), dbl, C.POINTER(pm_fourier), vp, vp, i64, i64,
                                             dbl, C.c_uint64, u32, vp, vp, vp]
    L.pm_forward_batched.argtypes = [vp, C.POINTER(pm_batch), u32, vp, vp, vp]
    L.pm_autotune_batched.argtypes = [vp, C.POINTER(pm_batch), u32, vp]
    L.pm_autotune_dirichlet.argtypes = [vp, C.POINTER(pm_field), dbl, dbl, C.POINTER(pm_dirichlet_data), vp, i64,
                                        i64, dbl, i64, C.c_uint64, u32, vp]
    L.pm_set_graph_mode.argtypes = [vp, C.c_int]
    L.pm_set_kernel_timing.argtypes = [vp, C.c_int]
    L.pm_sincos_turns.argtypes = [vp, vp, i64, vp, vp]
    L.pm_set_wait_limit.argtypes = [vp, i64]
    L.pm_last_kernel_ms.argtypes = [vp]
    L.pm_last_kernel_ms.restype = C.c_float
    L.pm_launch_count.argtypes = [vp]
    L.pm_launch_count.restype = i64
    L.pm_last_step_count.argtypes = [vp]
    L.pm_last_step_count.restype = i64
    L.pm_last_grid.argtypes = [vp]
    L.pm_last_grid.restype = i64
    L.pm_path_groups.argtypes = [vp, vp, i64, C.c_double, vp, vp, vp, vp]
    L.pm_forward_square_bvp.argtypes = [vp, vp, vp, i64, i64, C.c_double, i64, C.c_uint64, u32, vp, vp, vp, vp,
                                        C.POINTER(pm_path_opts)]
    L.pm_set_ctas_per_sm.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, C.c_int32]
    L.pm_set_refill_pairs.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, C.c_int32]
    L.pm_tuned_shape.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, vp, vp]
    _lib = L
    return L


def _check(rc):
    if rc < 0:
        raise PMError(rc, load().pm_last_error().decode())
    return rc


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Address of an array: numpy (host) or torch tensor (device or host)."""
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return a.ctypes.data


def _device(*arrays):
    dev = [a is not None and _is_torch(a) and a.is_cuda for a in arrays]
    present = [a is not None for a in arrays]
    if any(dev) and not all(d for d, p in zip(dev, present) if p):
        raise ValueError("mix of device and host arrays")
    return any(dev)


class Field:
    """Keeps the host arrays of a pm_field alive."""

    def __init__(self, K, u):
        self.u = np.ascontiguousarray(u, dtype=np.float64)
        self.s = pm_field(int(K), 0, self.u.ctypes.data_as(C.POINTER(C.c_double)))


class Fourier:
    def __init__(self, k, a, b):
        self.k = np.ascontiguousarray(np.asarray(k, dtype=np.int32).reshape(-1, 2))
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.s = pm_fourier(len(self.a), 0, self.k.ctypes.data_as(C.POINTER(C.c_int32)),
                            self.a.ctypes.data_as(C.POINTER(C.c_double)), self.b.ctypes.data_as(C.POINTER(C.c_double)))


class DirichletData:
    def __init__(self, R, quad, f_const, a, b):
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.s = pm_dirichlet_data(float(R), float(quad), float(f_const), len(self.a), 0,
                                   self.a.ctypes.data_as(C.POINTER(C.c_double)),
                                   self.b.ctypes.data_as(C.POINTER(C.c_double)))


def pm_version():
    return load().pm_version()


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def pm_create(device=0, stream=None):
    """stream: a cudaStream_t value (e.g. torch.cuda.Stream().cuda_stream); 0
    (torch's default stream) maps to cudaStreamLegacy; None lets the library
    create its own stream."""
    h = C.c_void_p()
    if stream == 0:
        stream = CUDA_STREAM_LEGACY
    _check(load().pm_create(C.byref(h), int(device), stream))
    return h


def pm_destroy(ctx):
    load().pm_destroy(ctx)


def pm_stream(ctx):
    return load().pm_stream(ctx)


def pm_sincos_turns(ctx, x, s, c):
    """sin and cos of 2 pi x (float32 CUDA tensors) as the tensor-core kernels form them."""
    return _check(load().pm_sincos_turns(ctx, _ptr(x), int(x.numel()), _ptr(s), _ptr(c)))


def pm_set_kernel_timing(ctx, on):
    return _check(load().pm_set_kernel_timing(ctx, int(bool(on))))


def pm_set_wait_limit(ctx, polls):
    """Test setting: the next forward / GEMM call's tensor-core waits give up
    after ``polls`` polls (0: at once); negative restores the full bound."""
    return _check(load().pm_set_wait_limit(ctx, int(polls)))


def pm_last_kernel_ms(ctx):
    return float(load().pm_last_kernel_ms(ctx))


def pm_launch_count(ctx):
    return int(load().pm_launch_count(ctx))


def pm_last_step_count(ctx):
    return int(load().pm_last_step_count(ctx))


def pm_last_grid(ctx):
    return int(load().pm_last_grid(ctx))


def pm_path_groups(x, t, dt):
    """The observation groups PM_SHARE_PATHS forms (host only) ->
    (group_of [n_obs], stream_of [n_obs], n_groups, steps_per_path)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 2)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1)
    n = len(t)
    assert x.shape[0] == n
    gof = np.empty(n, dtype=np.int32)
    sof = np.empty(n, dtype=np.int32)
    ng = C.c_int64()
    sp = C.c_int64()
    rc = load().pm_path_groups(x.ctypes.data, t.ctypes.data, n, float(dt), gof.ctypes.data, sof.ctypes.data,
                               C.byref(ng), C.byref(sp))
    if rc < 0:
        raise PMError(rc, "pm_path_groups: invalid arguments")
    return gof, sof, int(ng.value), int(sp.value)


def _opts(path_offset=0, instance=0, g_out=None, x_out=None):
    return pm_path_opts(int(path_offset), int(instance), 0, _ptr(g_out), _ptr(x_out))


def pm_forward_timedep(ctx, field: Field, kappa, theta0: Fourier, x, t, n_obs, M, dt, seed, flags, mean, var=None,
                       path_offset=0, instance=0, g_out=None, x_out=None):
    if _device(x, t, mean, var, g_out, x_out):
        flags |= PM_DEVICE_PTRS
    o = _opts(path_offset, instance, g_out, x_out)
    return _check(load().pm_forward_timedep(ctx, C.byref(field.s), float(kappa), C.byref(theta0.s), _ptr(x), _ptr(t),
                                            int(n_obs), int(M), float(dt), int(seed), int(flags), _ptr(mean),
                                            _ptr(var), C.byref(o)))


def pm_forward_dirichlet(ctx, field: Field, drift_scale, kappa, g: DirichletData, x, n_obs, M, dt, max_steps, seed,
                         flags, mean, var=None, exit_step=None, n_unexited=None, path_offset=0, instance=0,
                         g_out=None, x_out=None):
    if _device(x, mean, var, exit_step, n_unexited, g_out, x_out):
        flags |= PM_DEVICE_PTRS
    o = _opts(path_offset, instance, g_out, x_out)
    return _check(load().pm_forward_dirichlet(ctx, C.byref(field.s), float(drift_scale), float(kappa), C.byref(g.s),
                                              _ptr(x), int(n_obs), int(M), float(dt), int(max_steps), int(seed),
                                              int(flags), _ptr(mean), _ptr(var), _ptr(exit_step), _ptr(n_unexited),
                                              C.byref(o)))


class pm_diffusion_forcing(C.Structure):
    _fields_ = [("s0", C.c_double * 2), ("s1", C.c_double * 2), ("milstein", C.c_int32), ("n_src", C.c_int32),
                ("w", C.c_double), ("c", C.c_void_p), ("F", C.c_void_p)]


class DiffusionForcing:
    """Host description of pm_diffusion_forcing (keeps its arrays alive):
    sigma_i(x) = s0[i] + s1[i] x_i, the Milstein term when milstein, sources
    F[q] exp(-w |x - c_q|^2)."""

    def __init__(self, s0, s1, milstein=True, c=(), F=(), w=0.0):
        self.c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, 2))
        self.F = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(-1))
        assert self.c.shape[0] == self.F.shape[0]
        s0 = np.asarray(s0, dtype=np.float64).reshape(2)
        s1 = np.asarray(s1, dtype=np.float64).reshape(2)
        self.s = pm_diffusion_forcing((C.c_double * 2)(*s0), (C.c_double * 2)(*s1), int(bool(milstein)),
                                      int(self.F.shape[0]), float(w), self.c.ctypes.data if self.F.size else None,
                                      self.F.ctypes.data if self.F.size else None)


def pm_forward_dirichlet_general(ctx, field: Field, drift_scale, g: DirichletData, df: DiffusionForcing, x, n_obs, M,
                                 dt, max_steps, seed, flags, mean, var=None, exit_step=None, n_unexited=None,
                                 path_offset=0, instance=0, g_out=None, x_out=None):
    if _device(x, mean, var, exit_step, n_unexited, g_out, x_out):
        flags |= PM_DEVICE_PTRS
    o = _opts(path_offset, instance, g_out, x_out)
    return _check(load().pm_forward_dirichlet_general(ctx, C.byref(field.s), float(drift_scale), C.byref(g.s),
                                                      C.byref(df.s), _ptr(x), int(n_obs), int(M), float(dt),
                                                      int(max_steps), int(seed), int(flags), _ptr(mean), _ptr(var),
                                                      _ptr(exit_step), _ptr(n_unexited), C.byref(o)))


class pm_square_bvp(C.Structure):
    _fields_ = [("b", C.c_double * 2), ("kappa", C.c_double), ("w", C.c_double), ("g_cos", C.c_double),
                ("g_quad", C.c_double), ("n_src", C.c_int32), ("reserved", C.c_int32), ("c", C.c_void_p)]


class SquareBVP:
    """Host description of the optimal-forcing problem (keeps its arrays alive)."""

    def __init__(self, b, kappa, c, w, g_cos=1.0, g_quad=0.0):
        self.c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, 2))
        b = np.asarray(b, dtype=np.float64).reshape(2)
        self.s = pm_square_bvp((C.c_double * 2)(b[0], b[1]), float(kappa), float(w), float(g_cos), float(g_quad),
                               int(self.c.shape[0]), 0, self.c.ctypes.data if self.c.size else None)


def pm_forward_square_bvp(ctx, prob: SquareBVP, x, n_obs, M, dt, max_steps, seed, flags, mean, var=None,
                          exit_step=None, n_unexited=None, path_offset=0, instance=0, g_out=None):
    if _device(x, mean, var, exit_step, n_unexited, g_out):
        flags |= PM_DEVICE_PTRS
    o = _opts(path_offset, instance, g_out, None)
    return _check(load().pm_forward_square_bvp(ctx, C.byref(prob.s), _ptr(x), int(n_obs), int(M), float(dt),
                                               int(max_steps), int(seed), int(flags), _ptr(mean), _ptr(var),
                                               _ptr(exit_step), _ptr(n_unexited), C.byref(o)))


def pm_philox(ctx, ctr, key0, key1, n, out, flags=0):
    if _device(ctr, out):
        flags |= PM_DEVICE_PTRS
    return _check(load().pm_philox(ctx, _ptr(ctr), int(key0), int(key1), int(n), _ptr(out), int(flags)))


def pm_normals(ctx, seed, b, j, i, n0, count, out, flags=0):
    if _device(out):
        flags |= PM_DEVICE_PTRS
    return _check(load().pm_normals(ctx, int(seed), int(b), int(j), int(i), int(n0), int(count), _ptr(out),
                                    int(flags)))


def pm_velocity(ctx, field: Field, x, npts, v, flags=0):
    if _device(x, v):
        flags |= PM_DEVICE_PTRS
    return _check(load().pm_velocity(ctx, C.byref(field.s), _ptr(x), int(npts), _ptr(v), int(flags)))


def pm_forward_timedep_noalloc(field: Field, kappa, theta0: Fourier, x, t, n_obs, M, dt, seed, flags, mean, var=None,
                               stream=None):
    """Allocation-free time-dependent map: device tensors only, scratch from the
    library's fixed device array (see include/pm.h)."""
    return _check(load().pm_forward_timedep_noalloc(C.byref(field.s), float(kappa), C.byref(theta0.s), _ptr(x),
                                                    _ptr(t), int(n_obs), int(M), float(dt), int(seed), int(flags),
                                                    _ptr(mean), _ptr(var), stream))


class Batch:
    """Keeps the arrays of a pm_batch alive.  ``instances`` is a list of dicts with
    keys kind, u, kappa, dt, row0, n_obs, M, seed (and drift_scale, max_steps for
    Dirichlet instances; stream, default the instance's position); u may be numpy
    (host) or CUDA tensors (device)."""

    def __init__(self, K, instances, x, t, theta0: Fourier = None, disk: DirichletData = None):
        self.keep = [x, t, theta0, disk]
        arr = (pm_instance * len(instances))()
        for q, d in enumerate(instances):
            u = d["u"]
            if not _is_torch(u):
                u = np.ascontiguousarray(u, dtype=np.float64)
            self.keep.append(u)
            arr[q] = pm_instance(int(d["kind"]), int(d.get("stream", q)), _ptr(u), float(d["kappa"]), float(d["dt"]),
                                 float(d.get("drift_scale", 1.0)), int(d.get("max_steps", 0)), int(d["row0"]),
                                 int(d["n_obs"]), int(d["M"]), int(d["seed"]))
        self.arr = arr
        self.device = _device(x, t, *[d["u"] for d in instances])
        n_rows = (x.shape[0] if hasattr(x, "shape") else len(x))
        self.s = pm_batch(int(K), len(instances), arr, C.pointer(theta0.s) if theta0 is not None else None,
                          C.pointer(disk.s) if disk is not None else None, _ptr(x), _ptr(t), int(n_rows))


def pm_forward_batched(ctx, batch: Batch, flags, mean, var=None, n_unexited=None):
    if batch.device or _device(mean, var, n_unexited):
        flags |= PM_DEVICE_PTRS
    return _check(load().pm_forward_batched(ctx, C.byref(batch.s), int(flags), _ptr(mean), _ptr(var),
                                            _ptr(n_unexited)))


def pm_set_graph_mode(ctx, on):
    return _check(load().pm_set_graph_mode(ctx, int(bool(on))))


def pm_autotune_batched(ctx, batch: Batch, flags):
    """Times the batched call for every CTAs-per-SM candidate; returns the fastest (kept in ctx)."""
    if batch.device:
        flags |= PM_DEVICE_PTRS
    best = C.c_int32()
    _check(load().pm_autotune_batched(ctx, C.byref(batch.s), int(flags), C.byref(best)))
    return best.value


def pm_autotune_dirichlet(ctx, field: Field, drift_scale, kappa, g: DirichletData, x, n_obs, M, dt, max_steps, seed,
                          flags):
    """Times the Dirichlet call for every CTAs-per-SM candidate; returns the fastest (kept in ctx)."""
    if _device(x):
        flags |= PM_DEVICE_PTRS
    best = C.c_int32()
    _check(load().pm_autotune_dirichlet(ctx, C.byref(field.s), float(drift_scale), float(kappa), C.byref(g.s), _ptr(x),
                                        int(n_obs), int(M), float(dt), int(max_steps), int(seed), int(flags),
                                        C.byref(best)))
    return best.value


def pm_set_ctas_per_sm(ctx, kind, K, flags, ctas_per_sm):
    return _check(load().pm_set_ctas_per_sm(ctx, int(kind), int(K), int(flags), int(ctas_per_sm)))


def pm_set_refill_pairs(ctx, kind, K, flags, pairs):
    return _check(load().pm_set_refill_pairs(ctx, int(kind), int(K), int(flags), int(pairs)))


def pm_tuned_shape(ctx, kind, K, flags):
    """(CTAs per SM, refill pairs) in use for (kind, K, flags); 0 = not tuned or set."""
    a, b = C.c_int32(), C.c_int32()
    _check(load().pm_tuned_shape(ctx, int(kind), int(K), int(flags), C.byref(a), C.byref(b)))
    return a.value, b.value


class pm_train_opts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("weight_decay", C.c_float), ("lr_decay", C.c_float),
                ("shuffle_seed", C.c_uint64)]


def _declare_surrogate(L):
    vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
    L.pm_surrogate_create.argtypes = [vp, C.POINTER(vp), i32, i32, i32, C.c_uint64]
    L.pm_surrogate_destroy.argtypes = [vp]
    L.pm_surrogate_destroy.restype = None
    L.pm_surrogate_set_params.argtypes = [vp, vp] + [vp] * 6
    L.pm_surrogate_get_params.argtypes = [vp, vp] + [vp] * 6
    L.pm_surrogate_gradients.argtypes = [vp, vp, vp, vp, i64, vp] + [vp] * 6
    L.pm_surrogate_train.argtypes = [vp, vp, vp, vp, i64, C.POINTER(pm_train_opts), u32, vp]
    L.pm_surrogate_infer.argtypes = [vp, vp, vp, i64, vp, u32]
    L.pm_surrogate_input_gradient.argtypes = [vp, vp, vp, vp, i64, vp, u32]
    L.pm_surrogate_save.argtypes = [vp, vp, C.c_char_p]
    L.pm_surrogate_load.argtypes = [vp, C.POINTER(vp), C.c_char_p]
    L.pm_gemm_bf16.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, vp, i32]


def _slib():
    L = load()
    if not getattr(L, "_surrogate_declared", False):
        _declare_surrogate(L)
        L._surrogate_declared = True
    return L


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def pm_surrogate_create(ctx, n_in, n_hidden, n_out, seed=0):
    h = C.c_void_p()
    _check(_slib().pm_surrogate_create(ctx, C.byref(h), int(n_in), int(n_hidden), int(n_out), int(seed)))
    return h


def pm_surrogate_destroy(net):
    _slib().pm_surrogate_destroy(net)


def pm_surrogate_set_params(ctx, net, W1, b1, W2, b2, W3, b3):
    arrs = [_f32(a) for a in (W1, b1, W2, b2, W3, b3)]
    return _check(_slib().pm_surrogate_set_params(ctx, net, *[a.ctypes.data for a in arrs]))


def pm_surrogate_get_params(ctx, net, n_in, n_hidden, n_out):
    out = [np.empty((n_hidden, n_in), np.float32), np.empty(n_hidden, np.float32),
           np.empty((n_hidden, n_hidden), np.float32), np.empty(n_hidden, np.float32),
           np.empty((n_out, n_hidden), np.float32), np.empty(n_out, np.float32)]
    _check(_slib().pm_surrogate_get_params(ctx, net, *[a.ctypes.data for a in out]))
    return out


def pm_surrogate_gradients(ctx, net, U, T, n_in, n_hidden, n_out):
    U, T = _f32(U), _f32(T)
    loss = np.zeros(1, np.float32)
    out = [np.empty((n_hidden, n_in), np.float32), np.empty(n_hidden, np.float32),
           np.empty((n_hidden, n_hidden), np.float32), np.empty(n_hidden, np.float32),
           np.empty((n_out, n_hidden), np.float32), np.empty(n_out, np.float32)]
    _check(_slib().pm_surrogate_gradients(ctx, net, U.ctypes.data, T.ctypes.data, U.shape[0], loss.ctypes.data,
                                          *[a.ctypes.data for a in out]))
    return float(loss[0]), out


def pm_surrogate_train(ctx, net, U, Y, epochs, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, shuffle_seed=0,
                       weight_decay=0.0, lr_decay=1.0):
    dev = _device(U, Y)
    if not dev:
        U, Y = _f32(U), _f32(Y)
    N = U.shape[0]
    o = pm_train_opts(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                      float(lr_decay), int(shuffle_seed))
    hist = np.zeros(int(epochs), np.float32)
    _check(_slib().pm_surrogate_train(ctx, net, _ptr(U), _ptr(Y), int(N), C.byref(o),
                                      PM_DEVICE_PTRS if dev else 0, hist.ctypes.data))
    return hist


def pm_surrogate_infer(ctx, net, U, Y, flags=0):
    if _device(U, Y):
        flags |= PM_DEVICE_PTRS
    return _check(_slib().pm_surrogate_infer(ctx, net, _ptr(U), int(U.shape[0]), _ptr(Y), int(flags)))


def pm_surrogate_input_gradient(ctx, net, U, dY, dU, flags=0):
    """dU[b] = J(U[b])^T dY[b] for every row b (vector-Jacobian product of the
    network at its input)."""
    if _device(U, dY, dU):
        flags |= PM_DEVICE_PTRS
    else:
        U, dY = _f32(U), _f32(dY)
        assert dU.dtype == np.float32 and dU.flags["C_CONTIGUOUS"]
    return _check(_slib().pm_surrogate_input_gradient(ctx, net, _ptr(U), _ptr(dY), int(U.shape[0]), _ptr(dU),
                                                      int(flags)))


def pm_surrogate_save(ctx, net, path):
    return _check(_slib().pm_surrogate_save(ctx, net, str(path).encode()))


def pm_surrogate_load(ctx, path):
    h = C.c_void_p()
    _check(_slib().pm_surrogate_load(ctx, C.byref(h), str(path).encode()))
    return h


def pm_gemm_bf16(ctx, A, lda, B, ldb, M, N, K, C_out, ldc):
    return _check(_slib().pm_gemm_bf16(ctx, _ptr(A), int(lda), _ptr(B), int(ldb), int(M), int(N), int(K),
                                       _ptr(C_out), int(ldc)))


class pm_pcn_config(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("K", C.c_int32), ("beta", C.c_double), ("sigma", C.c_double),
                ("seed", C.c_uint64), ("n_obs", C.c_int64), ("y", C.c_void_p), ("A", C.c_void_p),
                ("kappa", C.c_double), ("dt", C.c_double), ("M", C.c_int64), ("path_seed", C.c_uint64),
                ("theta0", C.POINTER(pm_fourier)), ("x", C.c_void_p), ("t", C.c_void_p), ("map_flags", C.c_uint32),
                ("reserved", C.c_uint32), ("screen_shift", C.c_void_p)]


class pm_pcn_stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("proposals", C.c_int64), ("stage1_accepts", C.c_int64),
                ("accepts", C.c_int64), ("forward_evals", C.c_int64), ("seconds", C.c_double),
                ("sq_jump", C.c_double)]


def _plib():
    L = _slib()
    if not getattr(L, "_pcn_declared", False):
        vp = C.c_void_p
        L.pm_pcn_create.argtypes = [vp, C.POINTER(vp), C.POINTER(pm_pcn_config), vp, vp, vp]
        L.pm_pcn_run.argtypes = [vp, vp, C.c_int64, C.POINTER(pm_pcn_stats)]
        L.pm_pcn_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.pm_pcn_destroy.argtypes = [vp]
        L.pm_pcn_destroy.restype = None
        L._pcn_declared = True
    return L


class PCN:
    """pCN chains on the device (plain, or delayed acceptance when `screen` is given)."""

    def __init__(self, ctx, K, u0, y, sigma, beta, seed, A=None, theta0: Fourier = None, x=None, t=None, kappa=0.0,
                 dt=1e-3, M=1, path_seed=0, screen=None, screen_scale=None, tensor=False, screen_shift=None):
        self.ctx = ctx
        self.keep = [np.ascontiguousarray(y, dtype=np.float64), np.ascontiguousarray(u0, dtype=np.float64)]
        self.C, self.n_u = self.keep[1].shape
        A_ = np.ascontiguousarray(A, dtype=np.float64) if A is not None else None
        x_ = np.ascontiguousarray(x, dtype=np.float64) if x is not None else None
        t_ = np.ascontiguousarray(t, dtype=np.float64) if t is not None else None
        sc = _f32(screen_scale) if screen_scale is not None else None
        sh = np.ascontiguousarray(screen_shift, dtype=np.float64) if screen_shift is not None else None
        self.keep += [A_, x_, t_, sc, theta0, sh]
        cfg = pm_pcn_config(self.C, int(K), float(beta), float(sigma), int(seed), len(self.keep[0]),
                            self.keep[0].ctypes.data, A_.ctypes.data if A_ is not None else None, float(kappa),
                            float(dt), int(M), int(path_seed), C.pointer(theta0.s) if theta0 is not None else None,
                            x_.ctypes.data if x_ is not None else None, t_.ctypes.data if t_ is not None else None,
                            PM_TENSOR if tensor else 0, 0, sh.ctypes.data if sh is not None else None)
        self.h = C.c_void_p()
        _check(_plib().pm_pcn_create(ctx, C.byref(self.h), C.byref(cfg), self.keep[1].ctypes.data, screen,
                                     sc.ctypes.data if sc is not None else None))

    def run(self, n_steps):
        st = pm_pcn_stats()
        _check(_plib().pm_pcn_run(self.ctx, self.h, int(n_steps), C.byref(st)))
        return {k: getattr(st, k) for k, _ in pm_pcn_stats._fields_}

    def state(self):
        u = np.empty((self.C, self.n_u))
        phi = np.empty(self.C)
        s = np.empty(self.n_u)
        n = C.c_int64()
        _check(_plib().pm_pcn_state(self.ctx, self.h, u.ctypes.data, phi.ctypes.data, s.ctypes.data, C.byref(n)))
        return u, phi, s, n.value

    def close(self):
        if self.h:
            _plib().pm_pcn_destroy(self.h)
            self.h = None

"""Cross-check of Philox4x32-10 (Salmon et al., SC'11) against the cuRAND
library's Philox4_32_10 device generator.  cuRAND's mapping from
(seed, subsequence, draw index) to (key, counter) is not assumed: the test
tries every placement of the 64-bit draw index and subsequence in the four
counter words and both orders of the seed's halves in the key, requires that
exactly one placement reproduces cuRAND, and then checks thousands of draws
with that placement against the FP64 oracle's Philox and the library's own
(pm_philox)."""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests import _gpu

pytestmark = pytest.mark.gpu
pm = _gpu.pm

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def curand(tmp_path_factory):
    # The probe is test-only: built under pytest's temporary directory, never
    # beside the library's own build products.
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(HERE, "gpu_probes", "curand_philox_probe.cu")
    out = str(tmp_path_factory.mktemp("curand_probe") / "curand_philox_probe.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    src, "-o", out], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.curand_philox_draws.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint)]
    lib.curand_philox_draws.restype = ctypes.c_int
    return lib


@pytest.fixture(scope="module")
def c():
    h = _gpu.ctx()
    yield h
    pm.pm_destroy(h)


def draws(lib, seed, subsequence, n, offset=0):
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = lib.curand_philox_draws(seed, subsequence, offset, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)))
    assert rc == 0
    return out


def layouts():
    """(name, key(seed), counter(k, s)) for every placement of the words."""
    lo = lambda v: v & 0xFFFFFFFF
    hi = lambda v: (v >> 32) & 0xFFFFFFFF
    keys = {"seed lo, hi": lambda sd: (lo(sd), hi(sd)), "seed hi, lo": lambda sd: (hi(sd), lo(sd))}
    words = ["k_lo", "k_hi", "s_lo", "s_hi"]
    for kname, kf in keys.items():
        for perm in itertools.permutations(range(4)):
            def ctr(k, s, perm=perm):
                vals = {"k_lo": lo(k), "k_hi": hi(k), "s_lo": lo(s), "s_hi": hi(s)}
                return [vals[words[p]] for p in perm]
            yield f"key ({kname}), counter ({', '.join(words[p] for p in perm)})", kf, ctr


def test_curand_philox_mapping_by_probe_and_bit_exact(curand, orc, c):
    seeds = [0, 1, 0x0123456789ABCDEF, (2025 << 32) | 77]
    subs = [0, 1, 3, 1 << 40 | 5]
    samples = {(sd, s): draws(curand, sd, s, 8) for sd in seeds for s in subs}
    matches = []
    for name, kf, ctr in layouts():
        ok = True
        for (sd, s), got in samples.items():
            cs = np.array([ctr(k, s) for k in range(8)], dtype=np.uint32)
            if not np.array_equal(orc.philox(cs, kf(sd)), got):
                ok = False
                break
        if ok:
            matches.append((name, kf, ctr))
    assert len(matches) == 1, [m[0] for m in matches]
    name, kf, ctr = matches[0]
    print("cuRAND Philox4_32_10 layout:", name)
    # thousands of draws, three streams: cuRAND == oracle == the library's own Philox
    for sd, s in [(99, 0), (0xFEEDFACECAFEBEEF, 12345), (7, (1 << 63) + 3)]:
        n = 4096
        got = draws(curand, sd, s, n)
        cs = np.array([ctr(k, s) for k in range(n)], dtype=np.uint32)
        key = kf(sd)
        assert np.array_equal(orc.philox(cs, key), got), name
        mine = np.empty_like(cs)
        pm.pm_philox(c, cs, key[0], key[1], n, mine)
        assert np.array_equal(mine, got), name

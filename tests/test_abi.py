"""CPU checks of the C ABI library: it builds, loads, and exports every entry
point that include/pm.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_forward_maps():
    names = declared_functions()
    for n in ("pm_create", "pm_destroy", "pm_forward_timedep", "pm_forward_dirichlet", "pm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1808_10580_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_version():
    import paper_1808_10580_gb300 as pm
    pm.load()
    assert pm.pm_version() >= 10000


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1808_10580_gb300 as pm
    with pytest.raises(pm.PMError):
        pm.pm_create(0)


def test_header_is_plain_c():
    # The boundary is a C ABI: the header must compile as C11 on its own (no
    # C++ types, references, default arguments or overloads).  The source goes
    # to the compiler on standard input, so nothing is written.
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = '#include "pm.h"\nint main(void) { pm_ctx* c = 0; (void)c; return pm_version() > 0 ? 0 : 1; }\n'
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-x", "c", "-"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

"""Builds the C part of the CPU oracle (test infrastructure only) into
``oracle/_build/liboracle.so`` with gcc.  ``-ffp-contract=off`` stops the
compiler from fusing multiply-adds, so the oracle gives the same bits on
x86-64 and aarch64."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def library_path() -> str:
    return os.path.join(OUT_DIR, "liboracle.so")


def stale() -> bool:
    out = library_path()
    return (not os.path.exists(out)) or os.path.getmtime(out) < os.path.getmtime(SRC)


def build() -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build())

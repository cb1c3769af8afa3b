"""Compile the FP64 oracle (plain C, OpenMP when available) into a shared
library under oracle/_build/.  Test infrastructure only.

Usage: python oracle/build.py   (or oracle.build.build() from Python)
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sss_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _compile(flags):
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range", *flags,
           "-o", LIB + ".tmp", SRC, "-lm"]
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    r = _compile(["-fopenmp"])
    if r.returncode != 0:  # no OpenMP runtime: single-threaded oracle
        r = _compile([])
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

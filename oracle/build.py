"""Compile the CPU oracle into a shared library next to its source.

Plain gcc, no FMA contraction, no fast-math (the oracle's arithmetic must be
the IEEE float32/float64 operations written in ginterp_oracle.c, one rounding
per operation, on x86_64 and aarch64 alike), built twice: single-threaded, and
with OpenMP over the points of each pass.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ginterp_oracle.c")


def library_path(threaded: bool = False) -> str:
    return os.path.join(HERE, "libginterp_oracle_omp.so" if threaded else "libginterp_oracle.so")


def _build_one(threaded: bool, force: bool) -> str:
    out = library_path(threaded)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", *(["-fopenmp"] if threaded else []), SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Both builds of the oracle: the plain single-threaded one, and one with OpenMP
    that runs the points of each pass on several threads (identical results)."""
    _build_one(True, force)
    return _build_one(False, force)


if __name__ == "__main__":
    print(build(force=True))

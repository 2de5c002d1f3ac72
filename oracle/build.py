"""Compile the CPU oracle into a shared library next to its source.

Plain gcc, no FMA contraction, no fast-math (the oracle's arithmetic must be
the IEEE float32/float64 operations written in ginterp_oracle.c, one rounding
per operation, on x86_64 and aarch64 alike).
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ginterp_oracle.c")


def library_path() -> str:
    return os.path.join(HERE, "libginterp_oracle.so")


def build(force: bool = False) -> str:
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-Wno-unused-parameter", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))

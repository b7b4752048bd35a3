"""Build the FP64 CPU oracle (plain C) into oracle/_build/liboracle.so.

Test infrastructure: the oracle is only loaded by the tests, the smoke check
and the benchmark's CPU-baseline leg.  ``-ffp-contract=off`` keeps every
multiply and add separately rounded, so the oracle gives the same bits on
x86-64 and AArch64 hosts.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "glemur_oracle.c")
SRC_CS = os.path.join(HERE, "glemur_oracle_cstep.c")
HDR = os.path.join(HERE, "glemur_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(LIB) for p in (SRC, SRC_CS, HDR, __file__))
    if stale:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               "-Wall", "-Wextra", "-o", tmp, SRC, SRC_CS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

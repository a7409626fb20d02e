"""Compile the FP64 CPU oracle (test infrastructure) into oracle/libmbh_oracle.so.

Plain gcc, -O2, no fast-math and no FMA contraction, so the oracle keeps the
IEEE double semantics of its source; OpenMP only spreads independent templates
or walkers across threads.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "mbh_oracle.c"), os.path.join(HERE, "pt_oracle.c")]
LIB = os.path.join(HERE, "libmbh_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wno-unused-function", *SRCS, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

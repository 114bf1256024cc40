"""Builds the C part of the oracle (``o2.c``, ``o3.c``) into ``oracle/_o2.so``.

TEST INFRASTRUCTURE ONLY: compiling the checker is not using it; only tests,
the smoke check and the benchmark's CPU-baseline leg load the result.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "o2.c")
SRCS = [SRC, os.path.join(HERE, "o3.c")]
LIB = os.path.join(HERE, "_o2.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in SRCS):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, *SRCS])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

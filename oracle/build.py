"""Compile the FP64 oracle (test infrastructure) into ``oracle/liboracle.so``.

Plain gcc, portable flags only (the same source builds on x86_64 and aarch64);
``-ffp-contract=off`` keeps every FP32/FP64 operation a separately rounded IEEE
operation, which the tick quantisation relies on.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dode_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into the shared library ``out``."""
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", src, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    return compile_source(SRC, LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

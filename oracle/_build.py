"""Build the oracle's C part (TEST INFRASTRUCTURE ONLY).

Compiles oracle/raster.c into oracle/_oracle_raster.so with gcc. The flag
-ffp-contract=off matters: without it gcc may fuse multiply-adds on aarch64,
and the float32 visibility arithmetic would no longer be rounded one
operation at a time as the oracle's bit-exact contract states.
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "raster.c")
LIB = os.path.join(HERE, "_oracle_raster.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

"""Compile the oracle's C source into oracle/liboracle.so (test infrastructure only)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "raysplats_oracle.c")


def library_path() -> str:
    return os.path.join(HERE, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Build with gcc: FP64 arithmetic, no contraction, no fast-math (the FP32 ray and Morton
    sequences must round exactly as written).  Rebuilds when the source is newer."""
    out = library_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))

"""Build libraysplats.so (the CUDA library behind include/raysplats.h) for sm_103a.

Each .cu translation unit is compiled in parallel with nvcc, then linked into one shared
library in paper_2501_19196_gb300/_lib/.  No torch, no cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB_NAME = "libraysplats.so"
SOURCES = ["lbvh.cu", "render_fwd.cu", "render_bwd.cu", "render_bwd_depth.cu", "api.cu", "fixed_scratch.cu", "train.cu", "scene.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def library_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-Xptxas", "-warn-spills"] + list(extra)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link; skips the work when the library is newer than every source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    out = library_path()
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(HERE, "..", "include", "raysplats.h"), __file__]
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(p) for p in deps if os.path.exists(p))
        if os.path.getmtime(out) >= newest:
            return out
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra_flags)
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    logs = []
    for obj, log in results:
        objs.append(obj)
        logs.append(log)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    if verbose:
        sys.stdout.write("".join(logs))
    return out


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))

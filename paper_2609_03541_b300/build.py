"""Builds the BU-MBAR C-ABI library ``libbumbar.so`` in-tree with nvcc for
sm_103a (B300). Usage: ``python -m paper_2609_03541_b300.build``."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libbumbar.so")
ROOT = os.path.dirname(HERE)
SOURCES = ["common.cu", "lse.cu", "lse_regs.cu", "lse_smaj.cu", "lse_fact.cu", "sci_loop.cu", "binning.cu", "prep.cu", "hessian.cu", "hessian_tc.cu", "cholesky.cu", "api.cu", "noalloc.cu", "server.cu", "reweight.cu", "selftest.cu", "autotune.cu", "batch_loop.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs, cmds = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
        deps.append(os.path.join(ROOT, "include", "bumbar.h"))
        if not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(d) for d in deps):
            cmds.append([nvcc(), *ARCH, *FLAGS, *(extra or []), "-c", path, "-o", obj])
        objs.append(obj)
    # translation units compile independently: one nvcc per core
    workers = max(1, min(len(cmds), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as pool:
        for cmd in cmds:
            if verbose:
                print(" ".join(cmd), flush=True)
        for r in pool.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds):
            if verbose or r.returncode != 0:
                sys.stdout.write(r.stdout)
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                raise subprocess.CalledProcessError(r.returncode, r.args)
    cmd = [nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)

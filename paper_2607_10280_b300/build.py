"""Build the in-tree CUDA library ``libmpsano.so`` for B300 (sm_103a).

    python -m paper_2607_10280_b300.build [--force]

nvcc cross-compiles without a GPU.  The shared library is written next to this
file so that it travels with the source tree.
"""
from __future__ import annotations

import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libmpsano.so")
SOURCES = (["circuit_fp64_t1_c128.cu", "circuit_fp64_t1_c64.cu", "circuit_mixed_t1_c128.cu", "circuit_mixed_t1_c64.cu",
            "circuit_fp64_t1_c32.cu", "circuit_fp64_t1_c16.cu", "circuit_orth64_t1_c32.cu", "circuit_orth64_t1_c16.cu",
            "pauli_launch_sweep.cu", "pauli_launch.cu", "pauli_launch_large.cu", "pauli_launch_real.cu"]
           + [f"circuit_{p}_t0_c{c}.cu" for p in ("fp64", "mixed") for c in (64, 128)]
           + [f"circuit_{p}_t{t}_c{c}.cu" for p in ("mixed", "fp64", "orth64") for t in (0, 1) for c in (4, 8, 16, 32)
              if not (t == 1 and p != "mixed" and c >= 16)]
           + ["circuit_dispatch.cu", "ladder_mpo.cu", "mpsano.cu", "noalloc.cu", "train.cu"])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "mpsano.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every translation unit (in parallel) and link libmpsano.so."""
    if not force and up_to_date():
        return LIB
    obj_dir = os.path.join(HERE, "_build")
    os.makedirs(obj_dir, exist_ok=True)
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, *extra]
    # the slowest units come first; at most one compiler per core
    jobs = max(1, os.cpu_count() or 1)
    procs, objs, failed = [], [], []
    for src in SOURCES:
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [*common, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        while len([1 for _, pr in procs if pr.poll() is None]) >= jobs:
            time.sleep(0.2)
        procs.append((src, subprocess.Popen(cmd)))
    failed = [src for src, pr in procs if pr.wait() != 0]
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    link = [_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.run(link, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])

"""Build libamgdd.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_2601_04112_gb300.build [--force]

Each translation unit is compiled in parallel into _build/, then linked
into paper_2601_04112_gb300/libamgdd.so (CUDA runtime linked statically).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = ["csrc/api.cu", "csrc/cycle_kernels.cu", "csrc/multi_kernels.cu", "csrc/setup_kernels.cu",
           "csrc/aggregate_kernels.cu", "csrc/server.cu", "csrc/structure.cpp"]
HEADERS = ["csrc/internal.h", "csrc/structure.h"]
LIB = os.path.join(HERE, "libamgdd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
            "-I", os.path.join(HERE, "csrc")]


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = nvcc_path()
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    hdr = [os.path.join(HERE, h) for h in HEADERS] + [os.path.join(ROOT, "include", "amgdd.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        sp = os.path.join(HERE, src)
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < _newest([sp] + hdr):
            jobs.append([nvcc, *_flags(), "-c", sp, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
        for j, f in zip(jobs, futs):
            r = f.result()
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {j[-3]}:\n{r.stderr}")
    if force or jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", LIB, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

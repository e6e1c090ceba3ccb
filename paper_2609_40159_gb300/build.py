"""Builds the CUDA library in-tree: one nvcc job per translation unit (run in
parallel), then a shared link into ``libsptrsv_gb300.so`` next to this file.
Target: sm_103a only."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsptrsv_gb300.so")
# bounds-checked debug variant: every gather index checked (SPTRSV_CHECKED)
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libsptrsv_gb300_checked.so")
SOURCES = ["api.cu", "analyze.cu", "prims.cu", "rewrite.cu", "solve.cu", "batch.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "sptrsv.h"))
    return files


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _variants(checked: bool):
    out = [(BUILD, LIB, [])]
    if checked:
        out.append((BUILD_CHECKED, LIB_CHECKED, ["-DSPTRSV_CHECKED"]))
    return out


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compiles the product library and (checked=True) its bounds-checked
    variant; every stale translation unit of both in one parallel pool.
    Returns the product library's path."""
    deps = _deps()
    headers = [d for d in deps if not d.endswith(".cu")]
    nvcc = _nvcc()
    jobs = []
    for bdir, _, extra in _variants(checked):
        os.makedirs(bdir, exist_ok=True)
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(bdir, src.replace(".cu", ".o"))
            if force or _stale(o, [s] + headers):
                jobs.append([nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for c, r in zip(jobs, res):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(c)}")
    for bdir, lib, _ in _variants(checked):
        objs = [os.path.join(bdir, s.replace(".cu", ".o")) for s in SOURCES]
        if force or jobs or _stale(lib, objs):
            tmp = lib + f".{os.getpid()}.tmp"
            r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
            if r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
                raise RuntimeError("nvcc link failed")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

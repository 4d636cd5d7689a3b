"""Build the nrd CUDA library (libnrd.so) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  No CMake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libnrd.so")
BUILD = os.path.join(HERE, "_build")
UNITS = ["hier.cu", "k_stencil.cu", "k_blas.cu", "k_pc.cu", "solver.cu", "capi.cu",
         "noalloc.cu", "peaks.cu", "k_vjp.cu", "k_time.cu", "regrid.cu",
         "nk_graph.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _compile(unit, verbose_ptxas=False):
    src = os.path.join(SRC, unit)
    obj = os.path.join(BUILD, unit + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-c", src, "-o", obj]
    if verbose_ptxas:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, r.stdout, r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    srcs = [os.path.join(SRC, u) for u in UNITS] + [os.path.join(SRC, "nrd_internal.h"),
                                                  os.path.join(HERE, "..", "include", "nrd.h")]
    if (not force and os.path.exists(OUT)
            and all(os.path.getmtime(OUT) >= os.path.getmtime(s) for s in srcs)):
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        res = list(ex.map(lambda u: _compile(u, verbose_ptxas), UNITS))
    objs = [o for o, _ in res]
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, OUT)
    if verbose_ptxas:
        for u, (_, log) in zip(UNITS, res):
            print("==", u, "\n", log)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))

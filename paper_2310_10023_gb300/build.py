"""Build libbbs.so (the CUDA library behind include/bbs.h) in-tree for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel and linked
into paper_2310_10023_gb300/libbbs.so.  Host code is compiled without FMA
contraction and device code with -fmad=false, because the voxel keys are
floors of FP32 / FP64 expressions whose rounding must be reproducible.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libbbs.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def cflags(extra=()):
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math,-Wall",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _needs(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "bbs.h")]
    jobs = []
    for s in srcs:
        obj = os.path.join(BUILD, os.path.basename(s) + ".o")
        if _needs(obj, [s, *headers]):
            jobs.append((s, obj))
    cc = nvcc()

    def one(job):
        s, obj = job
        cmd = [cc, *cflags(extra), "-c", s, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for out in ex.map(one, jobs):
            if verbose and out:
                sys.stderr.write(out)
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([cc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def ptxas_report(src: str) -> str:
    """Registers / spills / shared memory of one translation unit (-Xptxas -v)."""
    r = subprocess.run([nvcc(), *cflags(), "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", os.devnull],
                       capture_output=True, text=True)
    return r.stderr


if __name__ == "__main__":
    print(build(verbose=True))

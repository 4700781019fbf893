"""Build ``libppn.so`` (sm_103a) in-tree with nvcc.

Each translation unit is compiled in parallel to an object under ``_build/``
and linked into ``paper_2505_21013_gb300/libppn.so`` with the CUDA runtime
linked statically.  Only one ``-gencode`` (compute_103a / sm_103a).
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libppn.so")
SOURCES = ["kernels.cu", "pcg.cu", "pcg_smem.cu", "pcg_sr.cu", "pcg_static.cu", "scene.cu", "server.cu"]
HEADERS = ["common.cuh", "tetmath.cuh", "eigclamp.cuh", "contact.cuh", "kernels.h", "scene.h", "driver.h", "pcg_common.cuh", "halo.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libppn.so")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
            "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")] + ARCH + list(extra)


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "ppn.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, s):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append([cc] + _flags(extra) + ["-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for log in ex.map(run, jobs):
            if ptxas_info and log:
                print(log, file=sys.stderr)
    if jobs or not os.path.exists(LIB):
        link = [cc, "-shared", "-cudart", "static"] + ARCH + objs + ["-o", LIB + ".tmp"]
        run(link)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))

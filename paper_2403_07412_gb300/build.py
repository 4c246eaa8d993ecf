"""Build ``libvecchia.so`` (the CUDA library behind include/vecchia.h) for sm_103a.

Each translation unit is compiled by nvcc in parallel and the objects are linked into
``paper_2403_07412_gb300/libvecchia.so``.  Host code is compiled with
``-ffp-contract=off`` so host-side squared distances are never fused.

``checked=True`` (or VECCHIA_CHECKED=1 in the environment) builds the bounds-checked
variant ``libvecchia_checked.so`` with -DVECCHIA_CHECKED: every index the kernels read
through is checked before use and a bad one is recorded in the error slot instead of
being dereferenced.  The Python binding loads that variant when VECCHIA_CHECKED=1.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libvecchia.so")
BUILD = os.path.join(HERE, "_build")
OUT_CHECKED = os.path.join(HERE, "libvecchia_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["matern.cu", "loglik.cu", "plan.cu", "peak.cu", "batched.cu", "bigblock.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def checked_requested() -> bool:
    return os.environ.get("VECCHIA_CHECKED", "") == "1"


def _flags(verbose_ptxas: bool, checked: bool = False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                "-I", os.path.join(HERE, "..", "include")]
    if checked:
        f += ["-DVECCHIA_CHECKED"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    deps.append(os.path.join(HERE, "..", "include", "vecchia.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool | None = None) -> str:
    if checked is None:
        checked = checked_requested()
    bdir, out = (BUILD_CHECKED, OUT_CHECKED) if checked else (BUILD, OUT)
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(bdir, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, src):
            jobs.append([cc, "-c", src, "-o", obj] + _flags(verbose_ptxas, checked))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose_ptxas or r.returncode:
                sys.stderr.write(r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if jobs or not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"], check=True)
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                checked=True if "--checked" in sys.argv else None))

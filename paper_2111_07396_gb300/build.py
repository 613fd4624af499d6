"""Build libssp.so (sm_103a) in-tree with nvcc.

Each translation unit is compiled in parallel, then linked into
``paper_2111_07396_gb300/libssp.so``.  Host code is compiled with
``-ffp-contract=off`` so that no host expression is fused differently on x86
and Arm.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libssp.so")
SOURCES = ["ssp_api.cu", "ssp_server.cu", "ssp_fp32.cu", "ssp_fp32_clamp.cu", "ssp_fp64.cu",
           "ssp_fp64_clamp.cu", "ssp_redo.cu", "ssp_redo_clamp.cu", "ssp_fp32_shared.cu",
           "ssp_fp64_shared.cu", "ssp_redo_shared.cu", "ssp_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr",
                   "-I", os.path.join(ROOT, "include"), *extra]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(ROOT, "include", f) for f in ("ssp.h", "ssp_peaks.h")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc(), *_flags(extra), "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(len(jobs)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for c, r in zip(jobs, results):
            if verbose or r.returncode:
                print(" ".join(c))
                print(r.stdout, r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {c[-3]}")
    if force or jobs or _stale(SO, objs):
        tmp = SO + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "--cudart=static", *objs, "-o", tmp],
                           capture_output=True, text=True)
        if r.returncode:
            print(r.stdout, r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

"""Builds the CUDA library libtvl1flow.so in-tree for sm_103a with nvcc (no cmake, no torch
extension machinery): one object per translation unit, compiled in parallel, then linked."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libtvl1flow.so")
OBJ = os.path.join(PKG, "_build")
SOURCES = ["tvl1_api.cu", "tvl1_serve.cu", "tvl1_step.cu", "tvl1_noalloc.cu", "k_pyramid.cu", "k_admm.cu", "k_admm_roll.cu", "k_admm_roll_f32.cu",
           "k_admm_roll_f16.cu", "k_admm_roll_bf16.cu", "k_admm_persist.cu", "k_admm_persist_f32.cu",
           "k_admm_persist_f16.cu", "k_admm_persist_bf16.cu", "k_resident.cu", "k_pdr.cu", "k_cp.cu",
           "k_reduce.cu", "k_probe.cu", "k_adapt.cu", "k_admm_tile.cu", "k_cp_tile.cu"]
HEADERS = ["tvl1_internal.h", "tvl1_device.cuh", "k_admm_roll.cuh", "k_admm_math.cuh", "k_pdr_math.cuh",
           "k_cp_math.cuh", "k_tile_cells.cuh", "k_admm_persist.cuh", "tvl1_plan.h", "tvl1_step.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(PKG, "..", "include", "tvl1flow.h")]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, f in zip(jobs, futs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(j))
    objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

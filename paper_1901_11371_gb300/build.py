"""Build libhb.so in-tree: g++ for the host construction, nvcc (sm_103a) for the kernels.

Translation units compile in parallel; the shared object lands next to this
file.  Usage: ``python -m paper_1901_11371_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["hb_kernels.cu", "hb_sweep.cu", "hb_sweep_f64.cu", "hb_sweep_f32n.cu", "hb_sweep_f32w.cu",
              "hb_sweep_mix.cu", "hb_api.cu", "hb_solver.cu", "hb_noalloc.cu", "hb_apply1.cu", "hb_tc.cu", "hb_sweep_cols.cu"]
CPP_SOURCES = ["hb_host.cpp", "hb_plan.cpp", "hb_tc_host.cpp", "hb_swsched.cpp"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _sources():
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "hb.h"))
    return hs


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _sources() + _headers() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_nvcc=None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", CSRC]
    jobs = []
    for s in CU_SOURCES:
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, s), "-o", obj]
        if extra_nvcc:
            cmd[1:1] = list(extra_nvcc)
        jobs.append((cmd, obj))
    for s in CPP_SOURCES:
        obj = os.path.join(BUILD, s.replace(".cpp", ".o"))
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", *inc, "-c", os.path.join(CSRC, s), "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([nvcc, "-shared", *ARCH, "-Xcompiler", "-fopenmp", "-o", tmp, *[o for _, o in jobs], "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

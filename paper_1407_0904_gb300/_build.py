"""Build libcoffee.so in-tree for sm_103a (nvcc for the kernels, g++ for host code).

Translation units are compiled in parallel; objects go to ``_build/`` and the shared
library to the package directory, where the Python binding loads it.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcoffee.so")

CU_SOURCES = ["api.cu", "k_fp64.cu", "k_tc.cu", "k_tc_staged.cu", "k_tc_burgers.cu", "k_tc_burgers_stream.cu", "k_bwd.cu", "noalloc.cu", "k_batch.cu",
              "k_csr.cu", "k_tc_csr.cu", "k_tc_burgers_res.cu",
              "k_prism.cu", "k_prism_burgers.cu", "k_prism_tc.cu", "k_peaks.cu", "host_pipeline.cu", "k_simt.cu",
              "k_tc_burgers_fact.cu"]
CPP_SOURCES = ["tabulate.cpp"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"] + GENCODE
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.exists(cand) or cand == "nvcc"):
            return cand
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(force=False, verbose=False, extra_nvcc=()):
    """Compile every translation unit and link libcoffee.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(PKG, "..", "include", f) for f in ("coffee.h", "coffee_peaks.h", "coffee_diag.h")] + [os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= t for p in deps if os.path.exists(p)):
            return LIB
    nvcc = _nvcc()
    jobs, objs = [], []
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s.replace(".cu", ".o"))
        jobs.append([nvcc] + NVCC_FLAGS + list(extra_nvcc) + ["-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    for s in CPP_SOURCES:
        o = os.path.join(BUILD, s.replace(".cpp", ".o"))
        jobs.append(["g++"] + CXX_FLAGS + ["-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    tmp = LIB + ".tmp%d" % os.getpid()
    _run([nvcc, "-shared"] + GENCODE + objs + ["-o", tmp])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_nvcc=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)

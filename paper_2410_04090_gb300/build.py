"""Build libjslam.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel, then linked into one shared
library next to this file.  Host code is compiled without floating-point
contraction so that the host-built tables are plain IEEE double results.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libjslam.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

CUDA_SOURCES = ["k_detect.cu", "k_pyca.cu", "k_orb_match.cu", "k_refine.cu", "k_fc_ablation.cu", "k_skipnet.cu", "jslam_api.cu", "pfa_static.cu"]
HOST_SOURCES = ["tables.cpp", "tune_cache.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _sources():
    return [os.path.join(CSRC, s) for s in CUDA_SOURCES + HOST_SOURCES] + \
           [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + \
           [os.path.join(INCLUDE, "jslam.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for s in CUDA_SOURCES:
        obj = os.path.join(BUILD, s + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", *common, "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-c", os.path.join(CSRC, s), "-o", obj]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for s in HOST_SOURCES:
        obj = os.path.join(BUILD, s + ".o")
        jobs.append((["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-fno-fast-math",
                      "-I", CSRC, "-I", INCLUDE, "-c", os.path.join(CSRC, s), "-o", obj], obj))
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose_ptxas:
        sys.stdout.write("".join(logs))
    tmp = LIB + f".tmp{os.getpid()}"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)

"""Build the in-tree shared library libh2star.so (host C++ + sm_103a CUDA).

    python -m paper_2309_14085_gb300.build_lib

Compiles the host construction with g++ (OpenMP, no floating-point
contraction so x86 and Arm hosts round identically) and the CUDA kernels with
nvcc for sm_103a only, in parallel, then links one shared library next to this
file.  No CMake, no torch extension machinery.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libh2star.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(verbose=False, ptxas_info=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I" + os.path.join(HERE, "..", "include"), "-I" + CSRC]
    host_flags = ["-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off"]
    jobs = []
    objs = []
    for src in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src + ".o")
        if src.endswith(".cpp"):
            jobs.append(["g++", "-c", path, "-o", obj] + host_flags + inc)
        elif src.endswith(".cu"):
            cmd = [nvcc, "-c", path, "-o", obj, ARCH, "-O3", "-lineinfo", "-std=c++17",
                   "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off", "--expt-relaxed-constexpr"] + inc
            if ptxas_info:
                cmd.append("-Xptxas=-v")
            jobs.append(cmd)
        else:
            continue
        objs.append(obj)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    _run([nvcc, "-shared", "-o", LIB + ".tmp"] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)

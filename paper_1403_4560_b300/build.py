"""Build libsgmc.so in-tree for sm_103a (B300) with nvcc and g++.

Usage: python -m paper_1403_4560_b300.build [--force] [--verbose]
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsgmc.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-fmad=false", "--expt-relaxed-constexpr", "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
             "-I", os.path.join(CUDA, "include")]


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _fingerprint() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode())
                h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    stamp = os.path.join(OBJ, "fingerprint")
    fp = _fingerprint()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and \
            open(stamp).read() == fp:
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    cu, cpp = _sources()
    jobs = []
    for f in cu:
        o = os.path.join(OBJ, f + ".o")
        jobs.append(([NVCC] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) +
                     ["-c", os.path.join(CSRC, f), "-o", o], o))
    for f in cpp:
        o = os.path.join(OBJ, f + ".o")
        jobs.append((["g++"] + CXX_FLAGS + ["-c", os.path.join(CSRC, f), "-o", o], o))
    # translation units compile in parallel
    with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(lambda j: subprocess.check_call(j[0]), jobs))
    objs = [o for _, o in jobs]
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-o", tmp] + objs +
                          ["-cudart", "static", "-lpthread", "-ldl", "-lrt"])
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(fp)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)

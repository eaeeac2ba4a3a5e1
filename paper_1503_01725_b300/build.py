"""Build liblsm.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

    python -m paper_1503_01725_b300.build [--force]

The PSL builder (psl_build.cu) is compiled with -fmad=false: its FP64 results
must be the correctly rounded value of each written operation so that the
integer particle counts of Eq. 3 are reproducible. The sampling and transport
kernels (transport.cu) flush FP32 denormals to zero (-ftz=true): no quantity
there is subnormal (energies, lengths and probabilities are far above 1e-38),
every other operation keeps its IEEE rounding, and the square roots and
divisions drop their denormal handling (per 1e7-history step: sampling 0.256
-> 0.248 ms, photon pass 0.452 -> 0.436 ms, electron pass 0.422 -> 0.397 ms,
with the same counters; full fast-math measured slower on the electron pass).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblsm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "--expt-relaxed-constexpr"]
SOURCES = {
    "api.cu": [],
    "psl_build.cu": ["-fmad=false"],
    "physics.cu": [],
    "transport.cu": ["-ftz=true"],
    "nnls.cu": [],
    "denoise.cu": [],
    "train.cu": [],
    "eval.cu": [],
    "pslfile.cu": [],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.exists(c) or c == "nvcc"):
            return c
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "lsm.h"))
    objs = []
    for src, extra in SOURCES.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", s, "-o", o]
        stamp = o + ".cmd"            # the flags an object was built with
        old = open(stamp).read() if os.path.exists(stamp) else ""
        if force or _stale(o, [s] + headers) or old != " ".join(cmd):
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            subprocess.check_call(cmd)
            with open(stamp, "w") as f:
                f.write(" ".join(c for c in cmd if c != "-Xptxas=-v"))
    if force or _stale(LIB, objs):
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart"])
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)

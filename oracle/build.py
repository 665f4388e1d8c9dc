"""Compile the FP64 CPU oracle (test infrastructure) into oracle/_build/.

Plain gcc, portable flags only (the same source builds on x86_64 and aarch64).
Two builds of the same source: liblbm_oracle.so (the parity build, -O2, one
thread) and liblbm_oracle_omp.so (-O3 with OpenMP over the rows of each
whole-field pass, used only to time the oracle on all host cores).  Both use
ISO C99, so no floating-point contraction, and give bitwise the same results.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_oracle.so")
LIB_OMP = os.path.join(OUT_DIR, "liblbm_oracle_omp.so")

_FLAGS = {LIB: ["-O2"], LIB_OMP: ["-O3", "-fopenmp"]}


def _build_one(lib, force):
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["gcc", *_FLAGS[lib], "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, omp: bool = False) -> str:
    """Build the parity library (or, with omp=True, the OpenMP timing build)
    if it is missing or older than its source; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    return _build_one(LIB_OMP if omp else LIB, force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build(force="--force" in sys.argv, omp=True))

"""Compile the FP64 oracle (plain C) into oracle/liboracle.so.

-ffp-contract=off keeps every FP32 decision rule free of fused multiply-add
so that it is bit-exact; the FP64 arithmetic is plain IEEE double.

build_openmp() compiles the same source with -fopenmp into
oracle/liboracle_omp.so: the multi-core CPU baseline that the benchmark
times beside the single-threaded oracle (never used as the oracle itself).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ed_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")

_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-mfpmath=sse", "-msse2", "-fPIC", "-shared",
          "-Wall", "-Wno-unused-function"]


def _compile(out, extra, force):
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    subprocess.check_call(["gcc"] + _FLAGS + extra + ["-o", out + ".tmp", SRC, "-lm"])
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    return _compile(LIB, ["-Wno-unknown-pragmas"], force)


def build_openmp(force: bool = False) -> str:
    return _compile(LIB_OMP, ["-fopenmp"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_openmp(force=True))

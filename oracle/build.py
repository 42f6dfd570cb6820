"""Compile the CPU oracle (plain C) into oracle/liboracle.so.

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg load the result; the CUDA library never does.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_num.c", "orc_mat.c", "orc_gemm.c", "orc_sampled.c", "orc_lu.c", "orc_api.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["orc.h", "build.py"]
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in deps)


def build(force: bool = False) -> str:
    if force or _stale():
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-Wall",
               "-Wno-unknown-pragmas", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

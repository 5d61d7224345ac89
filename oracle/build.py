"""Compile the CPU oracle (plain C, FP64, OpenMP) into a shared library.

Test infrastructure: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use the library this builds.  The GPU library never links it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fmm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liborc.so")

# -ffp-contract=off: no fused multiply-add, so every FP32 geometry step is one
# rounding, the same sequence an FP32 implementation without contraction uses.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fopenmp", "-Wall"]


def build_oracle(force: bool = False, src: str = SRC, lib: str = LIB) -> str:
    """Build the oracle library (default oracle/_build/liborc.so) if missing or stale."""
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(src)):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build_oracle(force=True))

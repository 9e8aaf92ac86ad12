"""Compile the FP64 CPU oracle (test infrastructure only) into oracle/_build/.

The oracle is plain C, built with -ffp-contract=off so that no multiply-add is
fused, and with OpenMP over chain groups.  Nothing here is part of the product
path; only the tests, the smoke check and the benchmark's CPU-baseline leg load
the library it produces.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libssoracle.so")
SRC = os.path.join(HERE, "ss_oracle.c")


def build(force: bool = False) -> str:
    """Build the oracle shared library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    hdr = os.path.join(HERE, "ss_oracle.h")
    newest = max(os.path.getmtime(SRC), os.path.getmtime(hdr))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

"""Compile the FP64 CPU oracle (test infrastructure only) into oracle/_build/.

The oracle is plain C, built with -ffp-contract=off so that no multiply-add is
fused, and with OpenMP over chain groups.  Nothing here is part of the product
path; only the tests, the smoke check and the benchmark's CPU-baseline leg load
the library it produces.

SS_ORACLE_LIB (environment): path of an already compiled oracle library to
load instead of building this one.  The mutation tests use it to run the pins
against copies of the oracle with a planted mistake.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libssoracle.so")
SRC = os.path.join(HERE, "ss_oracle.c")
HDR = os.path.join(HERE, "ss_oracle.h")


def compile_oracle(src: str, out: str, extra=()) -> str:
    """Compile one oracle source file (its directory must hold ss_oracle.h)."""
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-Wextra", *extra, "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Build the oracle shared library if it is missing or older than its source."""
    override = os.environ.get("SS_ORACLE_LIB")
    if override:
        return override
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    return compile_oracle(SRC, LIB)


COUNT_LIB = os.path.join(OUT_DIR, "libssoracle_ops.so")


def build_counting(force: bool = False) -> str:
    """The single-threaded operation-counting build (-DOR_COUNT_OPS, no OpenMP)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(COUNT_LIB) and os.path.getmtime(COUNT_LIB) >= newest:
        return COUNT_LIB
    tmp = COUNT_LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-Wall", "-Wextra", "-DOR_COUNT_OPS", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, COUNT_LIB)
    return COUNT_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

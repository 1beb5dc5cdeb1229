"""Compile the CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

The oracle is built with IEEE float semantics and no contraction of
multiply-adds, so its float32 ray/triangle test rounds every operation in the
order written."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build", "liboracle.so")


def build(force=False):
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= max(os.path.getmtime(src), os.path.getmtime(hdr)):
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tmp = OUT + f".tmp{os.getpid()}"
    compile_library(src, tmp)
    os.replace(tmp, OUT)
    return OUT


def compile_library(src, out):
    """gcc with the oracle's flags: one C file (next to its oracle.h) to a
    shared library."""
    cmd = ["gcc", "-O2", "-std=c99", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

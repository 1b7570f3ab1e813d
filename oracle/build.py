"""Compile the FP64 CPU oracle into oracle/liboracle.so (test infrastructure).

Run as ``python oracle/build.py`` or call ``build()``.  Builds with -ffp-contract=off so every
multiply and add in oracle.c rounds on its own, and with OpenMP over independent per-agent loops.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-ffp-contract=off", "-fPIC", "-shared",
           "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

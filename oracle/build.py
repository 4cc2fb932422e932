"""Compile the oracle's C core (oracle/smerf_oracle.c) into oracle/libsmerf_oracle.so.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain gcc, no GPU, no CUDA.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "smerf_oracle.c")
LIB = os.path.join(HERE, "libsmerf_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

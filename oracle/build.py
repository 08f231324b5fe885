"""Compile the FP64 CPU oracle (``lbm_oracle.c``) into ``liboracle.so``.

Test infrastructure only: the product library never uses this file.  The
shared object is built in place, next to the source, with gcc and OpenMP, and
with ``-ffp-contract=off`` so that no multiply-add is fused and the rounding
follows the order of operations written in the C source.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build ``liboracle.so`` if it is missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-D_DEFAULT_SOURCE", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

"""Build the CQRRPT oracle shared library (test infrastructure only).

Compiles ``cqrrpt_oracle.c`` into ``liboracle.so`` beside this file with
plain IEEE semantics: no fast-math and no implicit contraction of a*b+c into
a fused multiply-add (``-ffp-contract=off``); every fma is explicit in the
source.  OpenMP only parallelises loops whose iterations are independent, so
results do not depend on the thread count.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cqrrpt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

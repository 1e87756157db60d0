"""Build step for the CPU oracle (test infrastructure only).

Compiles ``pn_oracle.c`` into ``libpnoracle.so`` beside it with plain gcc:
``-O2 -ffp-contract=off`` so that every + and * is a separately rounded IEEE
operation, and OpenMP so that the timed CPU baseline can spread independent
orbits over the host cores.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pn_oracle.c")
HDR = os.path.join(HERE, "pn_oracle.h")
LIB = os.path.join(HERE, "libpnoracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or stale; return its path."""
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def build_variant(out: str, extra_flags) -> str:
    """Compile pn_oracle.c with other code-generation flags into `out` (for
    tests that compare two roundings of the same arithmetic, e.g. with
    multiply-adds contracted into FMAs)."""
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall"] + list(extra_flags) + \
          ["-o", out, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return out


if __name__ == "__main__":
    print(build(force=True))

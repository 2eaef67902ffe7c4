"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

Compiled with gcc, IEEE FP64 and no floating-point contraction so that the
x86 development host and the Arm GPU host produce identical bits.  OpenMP is
used when the compiler accepts it; results do not depend on the thread count
because every grid line is solved independently.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "aniso_oracle.c"), os.path.join(HERE, "aniso3d_oracle.c")]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS)):
        return LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall"]
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = base + ["-fopenmp"] + SRCS + ["-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: build single-threaded
        cmd = base + SRCS + ["-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

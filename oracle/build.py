"""Build the FP64 CPU oracle (test infrastructure) as a shared library next to its source.

Plain gcc, -O2, no fast-math and no floating-point contraction, so that x86-64 and aarch64
hosts produce the same bits; OpenMP over lattice rows (the result does not depend on the
thread count: every pass writes disjoint nodes and the reductions are serial).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mclbm_ref.c")
LIB = os.path.join(HERE, "libmclbm_ref.so")


def build(force: bool = False) -> str:
    """Compile oracle/mclbm_ref.c into oracle/libmclbm_ref.so (skipped when up to date)."""
    hdr = os.path.join(HERE, "mclbm_ref.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fopenmp", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

The oracle is the checker for the CUDA path: only the tests, the smoke check and
the benchmark's CPU-baseline leg load it.  Built with plain gcc, no
machine-specific flags and no FP contraction, so x86 and Arm hosts produce the
same bits.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sscn_ref.c")
LIB = os.path.join(HERE, "libsscn_ref.so")


def build(force: bool = False) -> str:
    """Compile oracle/sscn_ref.c into oracle/libsscn_ref.so; return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

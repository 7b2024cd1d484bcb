"""Build the FP64 CPU oracle (test infrastructure) as a shared library.

gcc -O2 -ffp-contract=off -fopenmp: no FMA contraction anywhere, so that the
tracer's crossing parameters are plain IEEE divisions and subtractions.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rt3d_oracle.c")
SRCS = [SRC, os.path.join(HERE, "rt3d_oracle_sph.c")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librt3d_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared library is missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and all(
            os.path.getmtime(LIB) >= os.path.getmtime(f) for f in SRCS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, *SRCS, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

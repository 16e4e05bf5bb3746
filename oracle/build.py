"""Compile the C oracle into ``oracle/_build/libcfd_oracle.so`` (plain gcc).

The flags keep every floating-point operation a separately rounded IEEE
double operation: no contraction into FMA, no fast-math.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cfd_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcfd_oracle.so")

BASE_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
              "-Wall", "-Wno-unknown-pragmas"]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        deps = [SRC, os.path.join(HERE, "cfd_oracle.h"), __file__]
        if os.path.getmtime(LIB) >= max(os.path.getmtime(p) for p in deps):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    for omp in (["-fopenmp"], []):
        cmd = ["gcc", *BASE_FLAGS, *omp, SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

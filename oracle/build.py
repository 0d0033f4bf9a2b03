"""Build the CPU oracle (test infrastructure) into oracle/_build/liboracle.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRC = [os.path.join(HERE, "f3r_oracle.cpp")]
DEPS = SRC + [os.path.join(HERE, "f3r_oracle.h")]

# ISO C++ mode plus -ffp-contract=off: no implicit multiply-add fusion; every
# fused multiply-add in the oracle is an explicit std::fma call.
FLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
         "-shared", "-fPIC", "-Wall"]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t_lib = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t_lib for s in DEPS):
            return LIB
    cmd = ["g++", *FLAGS, *SRC, "-o", LIB + ".tmp"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

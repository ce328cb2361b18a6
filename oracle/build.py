"""Compile the CPU oracle (test infrastructure only) into oracle/liboracle_ugkwp.so.

Plain g++, C++17, with floating-point contraction disabled so that every
operation the oracle writes is one IEEE-754 operation on any host.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle.cpp"]
LIB = os.path.join(HERE, "liboracle_ugkwp.so")
FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["omath.hpp", "dual.hpp", "ugkwp_oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in deps)


def build_oracle(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources."""
    if force or _stale():
        cmd = ["g++", *FLAGS, *[os.path.join(HERE, f) for f in SOURCES], "-o", LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))

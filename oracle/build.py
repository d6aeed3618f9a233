"""Builds the oracle shared library (test infrastructure only).

    python oracle/build.py

Compiles oracle/oracle_capi.cpp with g++ at -O2 and without floating-point
contraction, so that every a*b+c in the oracle rounds twice, as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liboracle.so")
SOURCES = ["oracle_capi.cpp", "mhd_oracle.hpp", "glm_oracle.hpp", "scalar.hpp"]


def needs_build():
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES)


def build(force=False):
    if not force and not needs_build():
        return SO
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-variable", "-Wno-unused-but-set-variable",
           os.path.join(HERE, "oracle_capi.cpp"), "-o", SO + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(SO + ".tmp", SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

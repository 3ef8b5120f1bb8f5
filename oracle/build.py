"""Build the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

Plain gcc, no target-specific flags, so the same command builds on x86-64
and on aarch64 hosts.  -ffp-contract=off keeps every multiply and add
separately rounded, as the oracle's source reads.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wb_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
COUNT_SRC = os.path.join(HERE, "count_ops.cpp")
COUNT_LIB = os.path.join(HERE, "liboracle_count.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "wb_oracle.h"))
    ):
        return LIB
    cmd = [
        os.environ.get("CC", "gcc"), "-O2", "-std=c11", "-ffp-contract=off",
        "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-Wall",
        SRC, "-o", LIB + ".tmp", "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def build_count(force: bool = False) -> str:
    """The operation-counting build of the same source (count_ops.cpp),
    single-threaded."""
    deps = [SRC, COUNT_SRC, os.path.join(HERE, "wb_oracle.h")]
    if not force and os.path.exists(COUNT_LIB) and os.path.getmtime(COUNT_LIB) >= max(
        os.path.getmtime(d) for d in deps
    ):
        return COUNT_LIB
    cmd = [
        os.environ.get("CXX", "g++"), "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
        "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas", "-I", HERE,
        COUNT_SRC, "-o", COUNT_LIB + ".tmp", "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(COUNT_LIB + ".tmp", COUNT_LIB)
    return COUNT_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

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


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

"""Compiles the FP64 CPU oracle (``lbmd_oracle.c``) into ``liblbmd_oracle.so``.

Test infrastructure: the library it builds is loaded only by the test suite,
the smoke check and the benchmark's CPU-baseline leg.

``-ffp-contract=off`` keeps the compiler from fusing multiplies and adds, so
the oracle's FP64 cell indices and pair distances are the plain IEEE
operation sequence written in the source on every host (gcc contracts by
default on aarch64).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbmd_oracle.c")
LIB = os.path.join(HERE, "liblbmd_oracle.so")


def build_oracle(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", LIB + ".tmp", SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))

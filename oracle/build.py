"""Compile the C oracle into oracle/lib/libtwofluid_oracle.so (gcc, OpenMP).

TEST INFRASTRUCTURE: built alongside the library, never used by the product path.
Flags: -O2, no fast-math and no FMA contraction, so the oracle rounds the
same way on x86-64 and aarch64.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libtwofluid_oracle.so")
SRC = [os.path.join(HERE, "twofluid_oracle.c")]
HDR = [os.path.join(HERE, "twofluid_oracle.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in SRC + HDR)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp] + SRC + ["-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

"""Compile the CPU oracle (test infrastructure) into oracle/_lib/liboracle.so.

Plain gcc, no build system.  -ffp-contract=off keeps every double expression
(the eps -> s bound, delta) evaluated exactly as written, without fused
multiply-adds, on x86-64 and on AArch64 alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_lib", "liboracle.so")
SRC = [os.path.join(HERE, "oracle.c")]
DEPS = SRC + [os.path.join(HERE, "netsimplex.inc")]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in DEPS)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-strict-aliasing", "-o", tmp] + SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

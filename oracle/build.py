"""Compile the FP64 oracle into ``oracle/_lib/liboracle.so``.

TEST INFRASTRUCTURE ONLY: the oracle checks the CUDA library; the product
path never loads it.

The oracle is built with ``-ffp-contract=off`` so that no multiply-add is
fused: the inside test of the re-discretisation must round exactly as the
source reads.  The host code is portable C (no intrinsics, no -march).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bloodlb_oracle.c")
OUT_DIR = os.path.join(HERE, "_lib")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(OUT) and os.path.getmtime(OUT) >= os.path.getmtime(SRC):
        return OUT
    tmp = OUT + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-D_DEFAULT_SOURCE", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

"""Compile the oracle's plain-C part (test infrastructure only) into oracle/_build/.

Run ``python -m oracle.build`` or call ``build()``; ``__graft_entry__.build()``
calls it so the checker exists on whichever machine runs the tests.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle_nbody.so")


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "nbody_ref.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(src):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps every multiply and add a separately rounded FP64 operation.
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lpthread", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

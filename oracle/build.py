"""Compile the C oracle into ``oracle/_liboracle.so`` with gcc (plain C, -O2).

Building the checker is not using it: ``__graft_entry__.build()`` calls this so
the oracle exists on every machine the tests run on.
"""
from __future__ import annotations

import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "_liboracle.so")
_LOCK = threading.Lock()  # threads of one process (the all-core CPU baseline) build once


def build(force: bool = False) -> str:
    with _LOCK:
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
            return LIB
        # a private temporary per process, then an atomic rename: concurrent
        # processes may each compile, and every rename installs a whole library
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                        "-std=c11", "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True))

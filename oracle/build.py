"""Compile the CPU oracle (plain C, FP64) into oracle/libslorc.so.

Test infrastructure: only the tests, the smoke check and the CPU-baseline
leg of the benchmark load the result."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sl_oracle.c")
SRCS = [SRC, os.path.join(HERE, "sl_learned.c"), os.path.join(HERE, "sl_eam_tab.c")]
DEPS = SRCS + [os.path.join(HERE, "orc_learned.h"), os.path.join(HERE, "orc_eam_tab.h")]
LIB = os.path.join(HERE, "libslorc.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(f) for f in DEPS):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *SRCS, "-o", tmp, "-lm"]
    # OpenMP only splits independent work (orc_set_threads); without it the
    # oracle runs on one thread with the same results
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

"""Build the C part of the oracle (libba_sparse.so) in-tree with gcc.

Test infrastructure only: the library is the block-sparse FP64 oracle loaded by
oracle/ba_sparse.py.  OpenMP is used when the compiler supports it; results do not depend
on the thread count.  -ffp-contract=off keeps every multiply and add separate, so the
library computes the same values on x86-64 and AArch64.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ba_sparse.c")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libba_sparse.so")
FLAGS = ["-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    cc = os.environ.get("CC") or shutil.which("gcc") or "cc"
    tmp = LIB + ".tmp"
    errors = []
    for extra in (["-fopenmp"], []):
        r = subprocess.run([cc, *FLAGS, *extra, SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
        errors.append(r.stderr)
    raise RuntimeError("oracle build failed:\n" + "\n".join(errors))


if __name__ == "__main__":
    print(build(force=True))

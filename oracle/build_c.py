"""Compile the oracle's C loops (oracle/o3_batch.c) into oracle/_build/.

Test infrastructure only: plain gcc with OpenMP, no CUDA, nothing shared with
the library. -ffp-contract=off keeps every multiply and add separate, so the
oracle rounds the same way on x86-64 and aarch64.
"""

from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "o3_batch.c")
LIB = os.path.join(BUILD, "libo3batch.so")


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle's C loops")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", SRC, "-o", tmp, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"oracle C build failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)

"""Builds the plain C part of the oracle (oracle/c/*.c) into oracle/liboracle.so with gcc.

Test infrastructure only: the library holds the float64 mass-action oracle used by the
tests and by the CPU-baseline leg of bench.py. It shares no code with the CUDA library.
"""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "c")
LIB = os.path.join(HERE, "liboracle.so")


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".c"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in sources() + [os.path.abspath(__file__)])


def build(force: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if not cc:
        raise RuntimeError("a C compiler (gcc) is required to build the oracle library")
    tmp = LIB + ".tmp"
    cmd = [cc, "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp,
           *sources(), "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

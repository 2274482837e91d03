"""Compile the CPU oracle (plain C) into oracle/_build/libpsco.so.

Test infrastructure: the oracle checks the CUDA path and is never linked into it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpsco.so")
SOURCES = [os.path.join(HERE, "psco.c")]


def build(force: bool = False) -> str:
    """Build the oracle shared library if it is missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in SOURCES + [os.path.join(HERE, "psco.h")])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    return compile_library(SOURCES, LIB)


def compile_library(sources, out):
    """Compile C sources into the shared library `out` with the oracle's flags
    (also used by tests that build a copy of the oracle with a planted mistake)."""
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp] + list(sources) + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

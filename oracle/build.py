"""Compiles the CPU oracle into oracle/_build/liboracle.so with gcc.

The oracle is test infrastructure: building it is part of building the checker,
it is never linked into the CUDA library.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SOURCES = [os.path.join(HERE, "pmc_oracle.c")]
HEADERS = [os.path.join(HERE, "pmc_oracle.h")]


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS)


def build_oracle(force: bool = False) -> str:
    """Builds the oracle library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-D_DEFAULT_SOURCE", "-o", tmp] + SOURCES + ["-lm"]
    # OpenMP spreads a batch's points over the host's cores when asked (orc_cache_set_threads);
    # without it the oracle still builds and runs on one thread
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build_oracle(force=True))

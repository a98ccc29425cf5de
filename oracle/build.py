"""Compile the CPU oracle into ``oracle/_build/libccmc_oracle.so``.

TEST INFRASTRUCTURE: the oracle is loaded only by the tests, the package's smoke
check and the CPU-baseline leg of the benchmark.  Built with gcc, one shared
object, ``-ffp-contract=off`` so that every floating-point step is rounded in
the order the source states (the threshold table must be bit-identical to the
library's, which is built the same way).
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libccmc_oracle.so")
SOURCES = ["ccmc_oracle.c", "exact_enum.c"]
HEADERS = ["ccmc_oracle.h"]


def _openmp_ok(cc: str) -> bool:
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads() < 0;}\n")
        r = subprocess.run([cc, "-fopenmp", src, "-o", os.path.join(td, "t")],
                           capture_output=True)
        return r.returncode == 0


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in SOURCES + HEADERS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    flags = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-Wall", "-Wextra"]
    if _openmp_ok(cc):
        flags.append("-fopenmp")
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, *flags, *[os.path.join(HERE, s) for s in SOURCES], "-o", tmp, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose=True))

"""Build ``libccmc.so`` in-tree (``paper_2301_11735_gb300/_build``) for sm_103a.

Nine translation units are compiled in parallel and linked into one shared
library that exports the C ABI of ``include/ccmc.h``:

* ``csrc/ccmc_phase.cu``   -- the colour-phase kernels (nvcc, sm_103a only);
* ``csrc/ccmc_map.cu``     -- the paper-faithful map mode's kernel;
* ``csrc/ccmc_maps.cpp``   -- host map generation (g++, host threads);
* ``csrc/ccmc_kernels.cu`` -- the other CUDA kernels (init, recount, packing);
* ``csrc/ccmc_api.cu``     -- host code of the C ABI (nvcc host pass);
* ``csrc/ccmc_noalloc.cu`` -- the recount entry point that allocates nothing;
* ``csrc/ccmc_peaks.cu``   -- measured shared-memory and L2 read bandwidth (diagnostics);
* ``csrc/ccmc_tables.cpp`` -- FP64 threshold tables (g++);
* ``csrc/ccmc_server.cpp`` -- the continuous-batching server (g++, a host thread).

All host code is compiled with ``-ffp-contract=off`` so the threshold tables
round exactly as written (an FMA would change the last bit of some entries).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libccmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC))


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = _sources() + [os.path.join(ROOT, "include", "ccmc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile the library if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    host = ["-Xcompiler", "-fPIC,-ffp-contract=off,-O2"]
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, *host]
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]
    jobs = {
        "ccmc_phase.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_phase.cu")],
        "ccmc_map.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_map.cu")],
        "ccmc_kernels.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_kernels.cu")],
        "ccmc_api.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_api.cu")],
        "ccmc_noalloc.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_noalloc.cu")],
        "ccmc_peaks.o": [nvcc, "-c", *common, os.path.join(CSRC, "ccmc_peaks.cu")],
        "ccmc_tables.o": [os.environ.get("CXX", "g++"), "-c", "-std=c++17", "-O2", "-fPIC",
                          "-ffp-contract=off", f"-I{cuda}/include",
                          os.path.join(CSRC, "ccmc_tables.cpp")],
        "ccmc_server.o": [os.environ.get("CXX", "g++"), "-c", "-std=c++17", "-O2", "-fPIC",
                          "-pthread", f"-I{cuda}/include", os.path.join(CSRC, "ccmc_server.cpp")],
        "ccmc_maps.o": [os.environ.get("CXX", "g++"), "-c", "-std=c++17", "-O2", "-fPIC",
                        "-pthread", os.path.join(CSRC, "ccmc_maps.cpp")],
    }
    procs = []
    for obj, cmd in jobs.items():
        cmd = cmd + ["-o", os.path.join(BUILD_DIR, obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((obj, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    failed = []
    for obj, p in procs:
        out, _ = p.communicate()
        if out and (verbose or ptxas_verbose or p.returncode):
            print(out, file=sys.stderr)
        if p.returncode:
            failed.append(obj)
    if failed:
        raise RuntimeError("libccmc build failed: " + ", ".join(failed))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    link = [nvcc, "-shared", *ARCH, "-o", tmp,
            *[os.path.join(BUILD_DIR, o) for o in jobs], "-lcudart_static", "-lrt", "-ldl",
            "-lpthread"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    subprocess.run(link, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, ptxas_verbose=True))

"""Compile libmpld (CUDA search kernels for sm_103a + host C++) in-tree.

The library is built with nvcc straight from ``csrc/`` into
``paper_2303_14335_gb300/_build/libmpld.so``; no torch extension machinery is
involved, because the ABI is plain C.  The integer-pipe throughput probe the
benchmark reports beside its roofline (``csrc/probe/``) goes into a separate
``_build/libmpld_probe.so``: measurement support, not part of the library.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmpld.so")
SOURCES = ["mpld_search.cu", "mpld_host.cpp", "mpld_serve.cpp"]
PROBE_SOURCES = [os.path.join("probe", "int_peak.cu")]
PROBE_LIB = os.path.join(OUT_DIR, "libmpld_probe.so")
HEADERS = ["mpld_internal.h", "mpld_problem.h", os.path.join("..", "..", "include", "mpld.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-Wall"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    for lib, srcs in ((LIB, SOURCES), (PROBE_LIB, PROBE_SOURCES)):
        if not os.path.exists(lib):
            return True
        t = os.path.getmtime(lib)
        deps = [os.path.join(CSRC, s) for s in srcs + HEADERS] + [__file__]
        if any(os.path.getmtime(d) > t for d in deps):
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libmpld.so if missing or out of date; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc, *ARCH, *COMMON, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd.insert(1, "-Xptxas=-v") if verbose else None
        subprocess.run(cmd, check=True, capture_output=not verbose)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES) + len(PROBE_SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES + PROBE_SOURCES))
    for lib, o in ((LIB, objs[:len(SOURCES)]), (PROBE_LIB, objs[len(SOURCES):])):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *o, "-lpthread"], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

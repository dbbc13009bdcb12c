"""Builds libkohler.so in place with nvcc (sm_103a only).

The library is compiled from the sources in ``csrc/`` into the package
directory, where the Python binding loads it.  Run ``python -m
paper_1707_05062_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libkohler.so")
SOURCES = ["kohler_api.cu", "kohler_server.cu", "kohler_segment.cu", "kohler_tune.cu"]
# measurement probes of the ceilings the strip pass runs into (bench.py's ceiling form)
PROBE_LIB = os.path.join(HERE, "libkohler_probe.so")
PROBE_SOURCES = ["kohler_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "kohler.h"))
    return files


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PROBE_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + list(extra)
    if verbose:
        common += ["-Xptxas", "-v"]
    procs, objs, pobjs = [], [], []
    for src in SOURCES + PROBE_SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        (pobjs if src in PROBE_SOURCES else objs).append(obj)
        procs.append(subprocess.Popen([nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + common))
    failed = [p.wait() for p in procs]
    if any(failed):
        raise RuntimeError("nvcc failed")
    for lib, parts in ((LIB, objs), (PROBE_LIB, pobjs)):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + parts + ["-lpthread"], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)

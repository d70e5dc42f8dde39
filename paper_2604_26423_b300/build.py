"""Builds libqaoa.so in-tree with nvcc for sm_103a (B300).

Usage: ``python -m paper_2604_26423_b300.build`` (or ``build_library()``).
The library is rebuilt when any source under ``csrc/`` or ``include/`` is newer.

Steps: the host-only generator ``csrc/gen_sigs.cpp`` (with the planner) is
built with g++ and writes ``csrc/pass_sigs.inc``, the round-signature sequences
of the specialised pass kernels; then every translation unit is compiled by
nvcc in parallel and the objects are linked into the shared library.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libqaoa.so")
SIGS = os.path.join(CSRC, "pass_sigs.inc")
GENERATOR = "gen_sigs.cpp"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _sources():
    srcs = glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp"))
    return sorted(s for s in srcs if os.path.basename(s) != GENERATOR)


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.join(CSRC, GENERATOR)]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def generate_sigs(verbose: bool = False) -> None:
    """Builds and runs gen_sigs; rewrites pass_sigs.inc only when its content changes."""
    cxx = os.environ.get("CXX", "g++")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "gen_sigs")
        out = os.path.join(tmp, "pass_sigs.inc")
        cmd = [cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(CSRC, GENERATOR),
               os.path.join(CSRC, "plan.cpp")]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        subprocess.check_call([exe, out], stdout=sys.stderr if verbose else subprocess.DEVNULL)
        with open(out) as f:
            new = f.read()
    old = open(SIGS).read() if os.path.exists(SIGS) else None
    if new != old:
        with open(SIGS, "w") as f:
            f.write(new)


def build_library(force: bool = False, verbose: bool = False, extra=None) -> str:
    if not force and not needs_build():
        return LIB
    generate_sigs(verbose)
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = tempfile.mkdtemp(prefix="qaoa_build_")
    try:
        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src) + ".o")
            cmd = [nvcc, *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, "-c", "-o", obj, src] + list(extra or [])
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            return obj

        srcs = _sources()
        with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
            objs = list(ex.map(compile_one, srcs))
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose=True))

"""Compile the CUDA library in-tree with nvcc for GB300 (sm_103a).

``python -m paper_1701_04685_gb300.build`` (or ``build()``) produces
``paper_1701_04685_gb300/_build/libffthomog.so``.  Sources are rebuilt when
any of them is newer than the library.  ``build(checked=True)`` produces
``libffthomog_checked.so``: the solver compiled with -DFH_CHECKED (index
checks in its kernels, see fftHomog.h), linked with the other objects of the
normal build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libffthomog.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libffthomog_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["solver.cu", "lattice.cpp", "noalloc.cu", "fno.cu"]
HEADERS = ["internal.hpp", "kernels.cuh", "fft.cuh", "cluster.cuh", "warprow.cuh", "linewarp.cuh", "colpass2.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    # every file of csrc/ counts, so that a header added later cannot be missed
    deps = [os.path.join(CSRC, f) for f in sorted(set(SOURCES + HEADERS) | set(os.listdir(CSRC)))]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [__file__]
    return any(os.path.getmtime(p) > t for p in deps)


def _compile_cuda(nvcc, src, obj, extra=()):
    return [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            *extra, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The checked library: solver.cu with -DFH_CHECKED, the other objects
    from the normal build."""
    if not force and not _stale(LIB_CHECKED) and not _stale():
        return LIB_CHECKED
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    obj = os.path.join(OUT_DIR, "solver_checked.o")
    cmd = _compile_cuda(nvcc, "solver.cu", obj, ("-DFH_CHECKED",))
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    # compiled alongside the normal build's objects
    proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    try:
        build(force=force, verbose=verbose)
    finally:
        out, _ = proc.communicate()
    if proc.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + out)
    objs = [obj] + [os.path.join(OUT_DIR, os.path.splitext(f)[0] + ".o") for f in SOURCES if f != "solver.cu"]
    tmp = LIB_CHECKED + ".tmp"
    r = subprocess.run([nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"], stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, LIB_CHECKED)
    return LIB_CHECKED


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    if checked:
        return build_checked(force=force, verbose=verbose)
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    procs = []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = _compile_cuda(nvcc, src, obj)
        if src.endswith(".cpp"):
            cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c",
                   os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    for p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + out)
        if verbose and out:
            print(out, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))

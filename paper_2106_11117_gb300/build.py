"""In-tree build of liblflts.so for sm_103a (nvcc + g++, no cmake).

The translation units compile in parallel; the CUDA runtime is linked
statically so the library only needs the driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblflts.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lflts.cu", "qoi_noalloc.cu", "mesh_prep.cpp"]
DEPS = SOURCES + ["kernels.cuh", "inner_tile.cuh", "inner_pair.cuh", "moving.cuh", "coarse_rc.cuh", "restride.cuh", "field_qoi.cuh", "adjoint.cuh", "mesh_prep.h"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblflts")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in DEPS] + [os.path.join(INCLUDE, "lflts.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile liblflts.so if a source changed; returns the library path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE] + (extra_flags or [])
    cmds, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc] + ARCH + ["-lineinfo", "-c", os.path.join(CSRC, src), "-o", obj] + common
        else:
            cmd = [nvcc, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", obj] + common
        cmds.append(cmd)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(c) + "\n" + out)
    tmp = LIB + ".tmp"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))

"""Build the CUDA shared library ``libhlbm.so`` in-tree for sm_103a.

Usage: ``python paper_2606_31707_b300/build.py [--force]`` (or ``build()``;
the package itself cannot be imported before the library exists).
Sources are compiled in parallel with nvcc and linked into the package
directory, next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhlbm.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["hlbm_primal.cu", "hlbm_adjoint.cu", "hlbm_krylov.cu", "hlbm_tangent.cu", "hlbm_capi.cu",
           "hlbm_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-v"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "hlbm.h"))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "hlbm.h"))
    return hs


def _obj_current(src: str, obj: str) -> bool:
    """The object exists and is newer than its source, every header and this script."""
    if not os.path.exists(obj):
        return False
    t = os.path.getmtime(obj)
    deps = [os.path.join(CSRC, src), os.path.abspath(__file__), *_headers()]
    return all(os.path.getmtime(p) <= t for p in deps if os.path.exists(p))


def _compile(src: str, log: bool) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    if _obj_current(src, obj):
        return obj
    cmd = [nvcc(), *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    if log:
        with open(os.path.join(BUILD, os.path.splitext(src)[0] + ".ptxas.txt"), "w") as fh:
            fh.write(r.stderr)
    return obj


def build(force: bool = False, log: bool = True) -> str:
    """Compile and link libhlbm.so if any source is newer; return its path."""
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for src in SOURCES:
            obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
            if os.path.exists(obj):
                os.remove(obj)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, log), SOURCES))
    tmp = OUT + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

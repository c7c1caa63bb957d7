"""Builds the CUDA library ``_build/liberi_gb300.so`` for sm_103a (GB300).

    python -m paper_2303_13632_gb300.build

The 55 canonical-class kernels are split over 16 translation units (one source file
compiled with -DERI_TU=k) that compile in parallel; objects are cached by a hash of the
sources and flags, so an unchanged tree links in well under a second.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liberi_gb300.so")
NUM_TU = 16

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _sources_digest() -> str:
    h = hashlib.sha1()
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h", ".inc")):
            with open(os.path.join(CSRC, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    with open(os.path.join(ROOT, "include", "eri.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:16]


def _units():
    units = [("eri_tables", "eri_tables.cu", []), ("eri_plan", "eri_plan.cu", []),
             ("eri_noalloc", "eri_noalloc.cu", []),
             ("eri_layout", "eri_layout.cu", []),
             ("eri_digest", "eri_digest.cu", []),
             ("eri_screen", "eri_screen.cu", []),
             ("eri_generic", "eri_generic.cu", [])]
    for k in range(NUM_TU):
        units.append((f"eri_classes_{k}", "eri_classes.cu", [f"-DERI_TU={k}"]))
    for k in range(4):
        units.append((f"eri_backward_{k}", "eri_backward.cu", [f"-DERI_BTU={k}"]))
    return units


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compiles (if needed) and returns the path of the shared library."""
    digest = _sources_digest()
    stamp = os.path.join(BUILD, "digest.txt")
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    objdir = os.path.join(BUILD, "obj_" + digest)
    os.makedirs(objdir, exist_ok=True)

    def compile_unit(u):
        name, src, defs = u
        obj = os.path.join(objdir, name + ".o")
        if os.path.exists(obj):
            return obj
        cmd = [exe, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        os.replace(obj + ".tmp", obj)
        return obj

    units = sorted(_units(), key=lambda u: 0 if u[0].startswith(("eri_classes", "eri_backward")) else 1)
    with ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        objs = list(ex.map(compile_unit, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    for name in os.listdir(BUILD):  # objects of older source trees
        if name.startswith("obj_") and name != "obj_" + digest:
            shutil.rmtree(os.path.join(BUILD, name), ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

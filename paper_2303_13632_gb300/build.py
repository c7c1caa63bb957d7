"""Builds the CUDA library ``_build/liberi_gb300.so`` for sm_103a (GB300).

    python -m paper_2303_13632_gb300.build

The 55 canonical-class kernels are split over 16 translation units (one source file
compiled with -DERI_TU=k) that compile in parallel.  Each object is cached under a hash of its
own source, the local headers it includes (followed recursively), its defines and the flags, so
an unchanged tree links in well under a second and a change to one file rebuilds only the units
that include it.
"""
from __future__ import annotations

import hashlib
import os
import re
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


_INCLUDE = re.compile(r'^\s*#\s*include\s*"([^"]+)"', re.M)


def _local_file(name: str) -> str | None:
    for d in (CSRC, os.path.join(ROOT, "include")):
        path = os.path.join(d, name)
        if os.path.exists(path):
            return path
    return None


def _unit_digest(src: str, defs) -> str:
    """Hash of a unit's source, every local header it includes (transitively), defines, flags."""
    h = hashlib.sha1()
    h.update(" ".join(ARCH + FLAGS + list(defs)).encode())
    seen, todo = set(), [os.path.join(CSRC, src)]
    while todo:
        path = todo.pop()
        if path in seen:
            continue
        seen.add(path)
        with open(path, "rb") as f:
            text = f.read()
        h.update(os.path.basename(path).encode())
        h.update(text)
        for inc in _INCLUDE.findall(text.decode("utf-8", "replace")):
            dep = _local_file(inc)
            if dep is not None:
                todo.append(dep)
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
    units = [(name, src, defs, _unit_digest(src, defs)) for name, src, defs in _units()]
    digest = hashlib.sha1(" ".join(u[0] + u[3] for u in units).encode()).hexdigest()[:16]
    stamp = os.path.join(BUILD, "digest.txt")
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    objdir = os.path.join(BUILD, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_unit(u):
        name, src, defs, h = u
        obj = os.path.join(objdir, f"{name}_{h}.o")
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

    # the slow class units first, so the pool's tail is short
    order = sorted(units, key=lambda u: 0 if u[0].startswith(("eri_classes", "eri_backward")) else 1)
    with ThreadPoolExecutor(max_workers=jobs or os.cpu_count() or 4) as ex:
        objs = dict(zip((u[0] for u in order), ex.map(compile_unit, order)))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *(objs[u[0]] for u in units)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    keep = {os.path.basename(o) for o in objs.values()}
    for name in os.listdir(objdir):  # objects of older sources
        if name.endswith(".o") and name not in keep:
            os.remove(os.path.join(objdir, name))
    for name in os.listdir(BUILD):  # per-tree object folders of the earlier layout
        if name.startswith("obj_"):
            shutil.rmtree(os.path.join(BUILD, name), ignore_errors=True)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

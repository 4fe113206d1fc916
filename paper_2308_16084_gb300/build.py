"""Build libp2m.so in-tree: nvcc for the CUDA translation units (sm_103a
only), g++ for the host builder, compiled in parallel and linked with nvcc.
No CMake."""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libp2m.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libp2m")
    return cand


def _sources():
    return {
        "kernels.cu": "cu", "certify.cu": "cu", "p2m_api.cu": "cu", "noalloc.cu": "cu",
        "flood.cu": "cu-nofma", "cells.cu": "cu-nofma", "pack.cu": "cu-nofma", "builder.cpp": "cpp",
    }


def _deps(path, seen=None):
    """The file and every header of this package it includes (quoted
    includes found in csrc/ or include/), recursively."""
    seen = set() if seen is None else seen
    if path in seen:
        return seen
    seen.add(path)
    with open(path) as f:
        text = f.read()
    for name in re.findall(r'^\s*#\s*include\s+"([^"]+)"', text, re.M):
        for d in (CSRC, os.path.join(ROOT, "include")):
            cand = os.path.join(d, name)
            if os.path.exists(cand):
                _deps(cand, seen)
                break
    return seen


def _obj_stale(src, obj):
    """An object is rebuilt when it is missing or older than its source, a
    header the source includes, or this script."""
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in _deps(os.path.join(CSRC, src)) | {__file__})


STAMP = os.path.join(OUT, "machine")


def _same_machine():
    """Objects are reused only on the machine type that compiled them (a
    copy of the tree may carry another architecture's objects)."""
    import platform
    try:
        with open(STAMP) as f:
            return f.read().strip() == platform.machine()
    except OSError:
        return False


def _stale():
    if not os.path.exists(LIB) or not _same_machine():
        return True
    t = os.path.getmtime(LIB)
    for src in _sources():
        obj = os.path.join(OUT, src + ".o")
        if _obj_stale(src, obj) or os.path.getmtime(obj) > t:
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the translation units whose objects are stale (all of them
    with force) and link the library when anything changed."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    force = force or not _same_machine()
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    extra = os.environ.get("P2M_EXTRA_NVCC_FLAGS", "").split()
    jobs, objs = [], []
    for src, kind in _sources().items():
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        if not force and not _obj_stale(src, obj):
            continue
        path = os.path.join(CSRC, src)
        if kind.startswith("cu"):
            # the device flooding and cells must round every double
            # operation on its own, as the host builder (-ffp-contract=off)
            # does
            nofma = ["-fmad=false"] if kind == "cu-nofma" else []
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-v" if verbose else "-O3", *nofma, *extra, *inc, "-c", path,
                   "-o", obj]
        else:
            cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off",
                   *inc, "-I", "/usr/local/cuda/include", "-c", path, "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max(1, len(jobs))) as ex:
        futs = [ex.submit(subprocess.run, c, capture_output=True, text=True) for c, _ in jobs]
        for (cmd, obj), f in zip(jobs, futs):
            r = f.result()
            if verbose and r.stderr:
                print(r.stderr)
            if r.returncode != 0:
                if os.path.exists(obj):
                    os.remove(obj)  # never link an object of an earlier source
                raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    import platform
    with open(STAMP, "w") as f:
        f.write(platform.machine() + "\n")
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv or "-v" in sys.argv, verbose="-v" in sys.argv))

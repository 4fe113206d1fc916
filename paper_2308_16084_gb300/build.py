"""Build libp2m.so in-tree: nvcc for the CUDA translation units (sm_103a
only), g++ for the host builder, compiled in parallel and linked with nvcc.
No CMake."""
from __future__ import annotations

import concurrent.futures as cf
import os
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


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
        [os.path.join(ROOT, "include", "p2m.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    extra = os.environ.get("P2M_EXTRA_NVCC_FLAGS", "").split()
    jobs = []
    for src, kind in _sources().items():
        obj = os.path.join(OUT, src + ".o")
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
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        futs = [ex.submit(subprocess.run, c, capture_output=True, text=True) for c, _ in jobs]
        for (cmd, _), f in zip(jobs, futs):
            r = f.result()
            if verbose and r.stderr:
                print(r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))

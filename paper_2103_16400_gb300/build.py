"""Builds libhexgpu.so in-tree with nvcc for sm_103a only.

    python -m paper_2103_16400_gb300.build

Each translation unit compiles in its own nvcc process (in parallel), then one
link step produces paper_2103_16400_gb300/_build/libhexgpu.so.  No cmake, no
torch extension machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhexgpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["plan.cpp", "capi.cpp", "ntt.cu", "ntt_f1.cu", "ntt_f2.cu", "ntt_i1.cu", "ntt_i2.cu",
           "ntt_f1s.cu", "ntt_f2s.cu", "ntt_i1s.cu", "ntt_i2s.cu", "ntt_tensor.cu", "ntt_tensor3.cu",
           "ntt_cluster_f.cu", "ntt_cluster_i.cu", "ntt_cluster_t.cu", "ntt_mul.cu", "ntt_muls.cu",
           "ntt_ctrow.cu",
           "eltwise.cu", "probe.cu",
           "batch.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhexgpu")


def _deps() -> list:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "hexgpu.h"))
    return files


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in _deps() + [src])


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I", os.path.join(ROOT, "include")] + (extra or [])
    if verbose:
        flags += ["-Xptxas", "-v"]

    def one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        if force or _stale(obj, os.path.join(CSRC, src)):
            cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            os.replace(obj + ".tmp", obj)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB)
                                               for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

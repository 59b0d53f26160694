"""Builds libgt.so (the CUDA library behind include/gt.h) in-tree for sm_103a.

The translation units compile in parallel with nvcc and link into
``paper_2009_07463_gb300/_build/libgt.so``. Rebuilds only when a source is newer.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libgt.so")
ARCH = "sm_103a"

SOURCES = ["scan.cu", "radix.cu", "build.cu", "bfs.cu", "batch.cu", "tune.cu", "serve.cu", "persist.cu", "capi.cu"]


def _deps() -> list[str]:
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return out


def nvcc_flags() -> list[str]:
    comp = ARCH.replace("sm_", "compute_")
    return ["-O3", "-std=c++17", f"-gencode=arch={comp},code={ARCH}", "-lineinfo",
            "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC,
            "--expt-relaxed-constexpr"]


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile libgt.so if any source changed; returns its path."""
    deps = _deps()
    if not force and os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    flags = nvcc_flags()

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = ["nvcc", *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["nvcc", "-shared", f"-gencode=arch={ARCH.replace('sm_', 'compute_')},code={ARCH}", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force=True))

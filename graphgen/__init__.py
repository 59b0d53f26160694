"""Seeded synthetic graph inputs: R-MAT (Graph500 initiator) and uniform edge tuples, BFS roots.

This module only makes inputs; it holds none of the BFS or edge-tree arithmetic. The CPU
oracle's tests and the GPU path both draw their inputs from it (host generator in
``gen_host.c``, device generator in ``gen_device.cu``, both defined in ``graphgen.h``), so a
seed names one graph on both sides.

Workload recipe (the paper's inputs, Sec. 6.1): R-MAT with A=0.57, B=C=0.19, D=0.05,
2^scale vertices, edgefactor * 2^scale tuples, ids scrambled by a keyed bijection;
self-loops and duplicate tuples are generated and left for the CSR build to drop.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_HOST_SO = os.path.join(_BUILD, "libgraphgen.so")
_DEV_SO = os.path.join(_BUILD, "libgraphgen_dev.so")
_lock = threading.Lock()
_host = None
_dev = None

GRAPH500_PPM = (570000, 190000, 190000)


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build_host() -> str:
    """Compile the host generator with gcc (idempotent)."""
    srcs = [os.path.join(_HERE, "gen_host.c"), os.path.join(_HERE, "graphgen.h")]
    if _stale(_HOST_SO, srcs):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _HOST_SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fvisibility=hidden",
                               "-o", tmp, srcs[0]])
        os.replace(tmp, _HOST_SO)
    return _HOST_SO


def build_device(arch: str = "sm_103a") -> str:
    """Compile the device generator with nvcc for sm_103a (idempotent)."""
    srcs = [os.path.join(_HERE, "gen_device.cu"), os.path.join(_HERE, "graphgen.h")]
    if _stale(_DEV_SO, srcs):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _DEV_SO + f".tmp{os.getpid()}"
        comp = arch.replace("sm_", "compute_")
        subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                               f"-gencode=arch={comp},code={arch}", "-lineinfo", "-o", tmp, srcs[0]])
        os.replace(tmp, _DEV_SO)
    return _DEV_SO


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            lib = ctypes.CDLL(build_host())
            i64, u64, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
            p = ctypes.c_void_p
            lib.gg_rmat_fill.argtypes = [u64, ctypes.c_int, i64, i64, u32, u32, u32, ctypes.c_int, p]
            lib.gg_uniform_fill.argtypes = [u64, i64, i64, i64, p]
            lib.gg_root_candidates.argtypes = [u64, i64, i64, i64, p]
            lib.gg_perm_fill.argtypes = [u64, ctypes.c_int, i64, i64, p]
            for f in (lib.gg_rmat_fill, lib.gg_uniform_fill, lib.gg_root_candidates, lib.gg_perm_fill):
                f.restype = None
            _host = lib
    return _host


def _dev_lib():
    global _dev
    with _lock:
        if _dev is None:
            lib = ctypes.CDLL(build_device())
            i64, u64, u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
            p = ctypes.c_void_p
            lib.gg_rmat_fill_device.argtypes = [u64, ctypes.c_int, i64, i64, u32, u32, u32, ctypes.c_int, p, p]
            lib.gg_uniform_fill_device.argtypes = [u64, i64, i64, i64, p, p]
            lib.gg_rmat_fill_device.restype = ctypes.c_int
            lib.gg_uniform_fill_device.restype = ctypes.c_int
            _dev = lib
    return _dev


def _parallel_fill(m: int, fill, threads: int | None = None) -> np.ndarray:
    out = np.empty((m, 2), dtype=np.int64)
    if m == 0:
        return out
    threads = threads or min(32, os.cpu_count() or 1)
    chunk = max(1 << 16, -(-m // threads))
    spans = [(b, min(chunk, m - b)) for b in range(0, m, chunk)]
    base = out.ctypes.data
    with ThreadPoolExecutor(max_workers=threads) as ex:  # ctypes releases the GIL
        list(ex.map(lambda s: fill(s[0], s[1], base + 16 * s[0]), spans))
    return out


def rmat_edges(scale: int, edgefactor: int = 16, seed: int = 1, ppm=GRAPH500_PPM, permute: bool = True,
               m: int | None = None) -> np.ndarray:
    """Host R-MAT tuples, int64 array of shape [m, 2], m = edgefactor * 2^scale by default."""
    if not 1 <= scale <= 31:
        raise ValueError("scale must be in [1, 31]")
    m = edgefactor * (1 << scale) if m is None else int(m)
    lib = _host_lib()
    a, b, c = ppm
    return _parallel_fill(m, lambda beg, cnt, ptr: lib.gg_rmat_fill(seed, scale, beg, cnt, a, b, c,
                                                                       int(permute), ptr))


def uniform_edges(n: int, m: int, seed: int = 1) -> np.ndarray:
    """Host uniform random tuples over [0, n), int64 [m, 2]."""
    if not 1 <= n <= (1 << 31):
        raise ValueError("n must be in [1, 2^31]")
    lib = _host_lib()
    return _parallel_fill(int(m), lambda beg, cnt, ptr: lib.gg_uniform_fill(seed, n, beg, cnt, ptr))


def perm_values(seed: int, scale: int) -> np.ndarray:
    """The id-scrambling map over [0, 2^scale) (tests check it is a bijection)."""
    n = 1 << scale
    out = np.empty(n, dtype=np.int64)
    _host_lib().gg_perm_fill(seed, scale, 0, n, out.ctypes.data)
    return out


def root_candidates(seed: int, n: int, begin: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    _host_lib().gg_root_candidates(seed, n, begin, count, out.ctypes.data)
    return out


def pick_roots(seed: int, n: int, k: int, degree: np.ndarray) -> np.ndarray:
    """The first k distinct root candidates (in candidate order) whose degree is >= 1.

    ``degree`` is the per-vertex degree in the cleaned graph (self-loops and duplicates
    dropped), from whichever side calls this.
    """
    degree = np.asarray(degree)
    nz = int(np.count_nonzero(degree))
    if nz < k:
        raise ValueError(f"graph has {nz} vertices of degree >= 1, fewer than the {k} roots asked for")
    picked: list[int] = []
    seen: set[int] = set()
    j = 0
    batch = max(4 * k, 1024)
    limit = 64 * n + 1024 * k
    while len(picked) < k:
        if j > limit:
            raise RuntimeError("root draw did not converge")
        cand = root_candidates(seed, n, j, batch)
        j += batch
        for c in cand.tolist():
            if degree[c] >= 1 and c not in seen:
                seen.add(c)
                picked.append(c)
                if len(picked) == k:
                    break
    return np.asarray(picked, dtype=np.int64)


def rmat_edges_device(out_ptr: int, scale: int, m: int, seed: int = 1, ppm=GRAPH500_PPM, permute: bool = True,
                      stream: int = 0) -> None:
    """Fill a device buffer of m * 2 int64 with the same tuples rmat_edges returns."""
    a, b, c = ppm
    rc = _dev_lib().gg_rmat_fill_device(seed, scale, 0, m, a, b, c, int(permute), out_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"gg_rmat_fill_device failed: cudaError {rc}")


def uniform_edges_device(out_ptr: int, n: int, m: int, seed: int = 1, stream: int = 0) -> None:
    rc = _dev_lib().gg_uniform_fill_device(seed, n, 0, m, out_ptr, stream)
    if rc != 0:
        raise RuntimeError(f"gg_uniform_fill_device failed: cudaError {rc}")

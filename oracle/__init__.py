"""CPU oracle for edge-tree BFS (arXiv 2009.07463): ctypes wrapper over ``oracle.c``.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. The GPU library never calls it and
the two share no code; the only common inputs come from ``graphgen``.

Functions (each cites the passage of the paper it follows, see ``oracle.c``):
  OracleGraph(edges, n)      simple undirected graph, sorted CSR (Sec. 5.1.1)
  OracleGraph.bfs(root)      levels + min-id parents, serial FIFO BFS (Alg. 1 top-down)
  OracleGraph.classify(mh)   vertex classes of Alg. 8 (Sec. 4.3)
  traversed_tuples(e, lvl)   Graph500 TEPS numerator
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CORE_INTERNAL, CORE_EDGE, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO = 0, 1, 2, 3, 4
CLASS_NAMES = ("CI", "CE", "TI", "TL", "VZ")


def build() -> str:
    """Compile oracle.c with gcc (idempotent)."""
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
    stale = not os.path.exists(_SO) or any(os.path.getmtime(s) > os.path.getmtime(_SO) for s in srcs)
    if stale:
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-fvisibility=hidden",
                               "-pthread", "-o", tmp, srcs[0]])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.or_graph_build.argtypes = [p, i64, i64, ctypes.c_int]
            lib.or_graph_build.restype = p
            lib.or_graph_free.argtypes = [p]
            lib.or_graph_free.restype = None
            lib.or_graph_n.argtypes = [p]
            lib.or_graph_n.restype = i64
            lib.or_graph_nnz.argtypes = [p]
            lib.or_graph_nnz.restype = i64
            lib.or_graph_csr.argtypes = [p, p, p]
            lib.or_graph_csr.restype = None
            lib.or_bfs.argtypes = [p, i64, p, p]
            lib.or_bfs.restype = ctypes.c_int
            lib.or_classify.argtypes = [p, ctypes.c_int, p, p, p]
            lib.or_classify.restype = ctypes.c_int
            lib.or_traversed_tuples.argtypes = [p, i64, p]
            lib.or_traversed_tuples.restype = i64
            _lib = lib
    return _lib


def _edges(edges) -> np.ndarray:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 2))
    return e


class OracleGraph:
    """Simple undirected graph of an edge-tuple list, held by the C oracle."""

    def __init__(self, edges, n: int, threads: int | None = None):
        self._lib = _load()
        e = _edges(edges)
        self.n = int(n)
        self.m = int(e.shape[0])
        threads = threads or min(64, os.cpu_count() or 1)
        h = self._lib.or_graph_build(e.ctypes.data, e.shape[0], self.n, int(threads))
        if not h:
            raise ValueError("oracle: vertex id out of range or out of memory")
        self._h = h
        self.nnz = int(self._lib.or_graph_nnz(h))

    def close(self):
        if self._h:
            self._lib.or_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def csr(self) -> tuple[np.ndarray, np.ndarray]:
        row = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        self._lib.or_graph_csr(self._h, row.ctypes.data, col.ctypes.data)
        return row, col[: self.nnz]

    def degree(self) -> np.ndarray:
        row, _ = self.csr()
        return np.diff(row)

    def bfs(self, root: int) -> tuple[np.ndarray, np.ndarray]:
        level = np.empty(self.n, dtype=np.int32)
        parent = np.empty(self.n, dtype=np.int32)
        rc = self._lib.or_bfs(self._h, int(root), level.ctypes.data, parent.ctypes.data)
        if rc != 0:
            raise ValueError(f"oracle bfs failed ({rc})")
        return level, parent

    def classify(self, mh: int = 0) -> tuple[np.ndarray, np.ndarray, int]:
        """(vertex_type[n] u8, peel_height[n] i32, height reached) of Alg. 8 with MH = mh."""
        vt = np.empty(self.n, dtype=np.uint8)
        ph = np.empty(self.n, dtype=np.int32)
        hr = ctypes.c_int32(0)
        rc = self._lib.or_classify(self._h, int(mh), vt.ctypes.data, ph.ctypes.data, ctypes.byref(hr))
        if rc != 0:
            raise MemoryError("oracle classify failed")
        return vt, ph, int(hr.value)


def traversed_tuples(edges, level: np.ndarray) -> int:
    e = _edges(edges)
    lv = np.ascontiguousarray(level, dtype=np.int32)
    return int(_load().or_traversed_tuples(e.ctypes.data, e.shape[0], lv.ctypes.data))

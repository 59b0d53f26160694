"""Edge-tree BFS on GB300 (arXiv 2009.07463): thin Python binding over libgt (include/gt.h).

The functions here carry the C-ABI's names and only marshal arguments: every step of the
path runs in the library's CUDA kernels. Buffers may be torch tensors (device or host),
numpy arrays (host) or raw integer pointers; streams are torch streams or raw handles.
There is no CPU fallback: if libgt.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import native

GT_OK, GT_EINVAL, GT_ENOMEM, GT_ETIMEOUT, GT_EBUSY, GT_EDEVICE, GT_ENOTSUP, GT_EIO = 0, -1, -2, -3, -4, -5, -6, -7
GT_SERVE_ADAPTIVE, GT_SERVE_BATCHED, GT_SERVE_SINGLE = 0, 1, 2
CORE_INTERNAL, CORE_EDGE, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO = 0, 1, 2, 3, 4


class gt_config(ctypes.Structure):
    _fields_ = [("mh", ctypes.c_int32), ("keep_plain", ctypes.c_int32)]


class gt_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "alpha", "beta", "td_warp_min", "td_cta_min", "td_grid_min", "bu_thread_scan", "blocks_per_sm",
        "force_direction", "launch_mode", "count_work", "time_kernels", "batch_alpha", "batch_beta", "bu_hub_first")]


class gt_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_core", ctypes.c_int64), ("nnz_core", ctypes.c_int64), ("n_class", ctypes.c_int64 * 5),
                ("mh", ctypes.c_int32), ("height", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class gt_level_info(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("direction", ctypes.c_int32), ("frontier", ctypes.c_int64),
                ("frontier_edges", ctypes.c_int64), ("unvisited_edges", ctypes.c_int64),
                ("discovered", ctypes.c_int64), ("examined", ctypes.c_int64), ("step_ms", ctypes.c_double)]


class gt_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("streams", ctypes.c_int32), ("max_batch_roots", ctypes.c_int32),
                ("window_us", ctypes.c_double), ("policy", ctypes.c_int32), ("join_levels", ctypes.c_int32)]


class gt_serve_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "batches", "inflight", "pending")] + \
               [(n, ctypes.c_double) for n in ("p50_us", "p99_us", "mean_us", "max_us", "qps")] + \
               [("device_bytes", ctypes.c_int64), ("joined", ctypes.c_int64), ("early", ctypes.c_int64)]


class GtError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'error'} (status {code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libgt (built in-tree on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = native.build()
            L = ctypes.CDLL(path)
            p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            sig = {
                "gt_config_default": (None, [p]),
                "gt_tuning_default": (None, [p]),
                "gt_graph_build": (ctypes.c_int, [p, i64, i64, p, p, p]),
                "gt_graph_free": (None, [p]),
                "gt_graph_stats": (ctypes.c_int, [p, p]),
                "gt_graph_vertex_type": (ctypes.c_int, [p, p, p]),
                "gt_graph_degree": (ctypes.c_int, [p, p, p]),
                "gt_graph_get_tuning": (ctypes.c_int, [p, p]),
                "gt_graph_set_tuning": (ctypes.c_int, [p, p]),
                "gt_bfs": (ctypes.c_int, [p, i64, p, p, p]),
                "gt_bfs_plain": (ctypes.c_int, [p, i64, p, p, p]),
                "gt_bfs_roots": (ctypes.c_int, [p, p, i32, p, p, p]),
                "gt_bfs_trace": (ctypes.c_int, [p, p, i32, p]),
                "gt_bfs_timing": (ctypes.c_int, [p, p]),
                "gt_bfs_csr_noalloc": (ctypes.c_int, [p, p, i64, i64, p, p, p]),
                "gt_bfs_batch": (ctypes.c_int, [p, i32, p, p, p, p, p]),
                "gt_autotune": (ctypes.c_int, [p, i32, ctypes.c_uint64, p, p]),
                "gt_serve_config_default": (None, [p]),
                "gt_serve_create": (ctypes.c_int, [p, p]),
                "gt_serve_add_graph": (ctypes.c_int, [p, p, p]),
                "gt_serve_submit": (ctypes.c_int, [p, i32, i64, p, p, p]),
                "gt_serve_poll": (ctypes.c_int, [p, ctypes.c_uint64, i32]),
                "gt_serve_get_stats": (ctypes.c_int, [p, p]),
                "gt_serve_reset_stats": (ctypes.c_int, [p]),
                "gt_serve_destroy": (ctypes.c_int, [p]),
                "gt_count_traversed": (ctypes.c_int, [p, i64, p, i64, p, p]),
                "gt_test_batch_barrier": (None, [ctypes.c_uint32, ctypes.c_uint32]),
                "gt_bfs_batch_work": (ctypes.c_int, [p, p]),
                "gt_test_fail_alloc": (None, [i32]),
                "gt_graph_save": (ctypes.c_int, [p, ctypes.c_char_p, p]),
                "gt_graph_load": (ctypes.c_int, [ctypes.c_char_p, p, p]),
                "gt_strerror": (ctypes.c_char_p, [ctypes.c_int]),
                "gt_last_error": (ctypes.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != GT_OK:
        raise GtError(rc, where, lib().gt_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _buf(x, count: int, what: str, dtype: str = "int32") -> int:
    """Pointer of a buffer, after checking that an array or tensor holds at least `count`
    contiguous entries of `dtype` (raw integer pointers are taken as given)."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if isinstance(x, np.ndarray):
        ok = x.dtype == np.dtype(dtype) and x.flags.c_contiguous and x.size >= count
    elif hasattr(x, "numel"):
        ok = str(x.dtype) == f"torch.{dtype}" and x.is_contiguous() and x.numel() >= count
    else:
        raise TypeError(f"{what}: cannot take a pointer of {type(x)}")
    if not ok:
        raise ValueError(f"{what}: need a contiguous {dtype} buffer of at least {count} entries")
    return _ptr(x)


def _out(x, count: int, what: str) -> int:
    """Pointer of an int32 output buffer of at least `count` entries (see _buf)."""
    return _buf(x, count, what)


def _stream(s) -> int:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _len_pairs(edges) -> int:
    shape = tuple(edges.shape)
    if len(shape) != 2 or shape[1] != 2:
        raise ValueError("edges must have shape [m, 2]")
    return int(shape[0])


def tuning_default() -> gt_tuning:
    t = gt_tuning()
    lib().gt_tuning_default(ctypes.byref(t))
    return t


class Graph:
    """A graph handle: device CSR, core CSR, edge-tree layout and traversal state."""

    def __init__(self, handle: int, n: int):
        self._h = handle
        self.n = n

    @property
    def handle(self) -> int:
        return self._h

    def free(self):
        if self._h:
            lib().gt_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        st = gt_stats()
        _check(lib().gt_graph_stats(self._h, ctypes.byref(st)), "gt_graph_stats")
        return {"n": st.n, "m": st.m, "nnz": st.nnz, "n_core": st.n_core, "nnz_core": st.nnz_core,
                "n_class": list(st.n_class), "mh": st.mh, "height": st.height, "device_bytes": st.device_bytes}

    def vertex_type(self, out=None, stream=None):
        out = np.empty(self.n, dtype=np.uint8) if out is None else out
        _check(lib().gt_graph_vertex_type(self._h, _ptr(out), _stream(stream)), "gt_graph_vertex_type")
        return out

    def degree(self, out=None, stream=None):
        out = np.empty(self.n, dtype=np.int32) if out is None else out
        _check(lib().gt_graph_degree(self._h, _ptr(out), _stream(stream)), "gt_graph_degree")
        return out

    def get_tuning(self) -> gt_tuning:
        t = gt_tuning()
        _check(lib().gt_graph_get_tuning(self._h, ctypes.byref(t)), "gt_graph_get_tuning")
        return t

    def set_tuning(self, t: gt_tuning | None = None, **kw):
        t = self.get_tuning() if t is None else t
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(lib().gt_graph_set_tuning(self._h, ctypes.byref(t)), "gt_graph_set_tuning")

    def bfs(self, root: int, parent=None, level=None, stream=None, plain: bool = False):
        """Levels and min-id parents from root; host numpy outputs when none are given."""
        if parent is None and level is None:
            parent = np.empty(self.n, dtype=np.int32)
            level = np.empty(self.n, dtype=np.int32)
        f = lib().gt_bfs_plain if plain else lib().gt_bfs
        _check(f(self._h, int(root), _out(parent, self.n, "parent"), _out(level, self.n, "level"), _stream(stream)),
               "gt_bfs_plain" if plain else "gt_bfs")
        return parent, level

    def bfs_roots(self, roots, parents, levels, stream=None):
        """gt_bfs_roots: one edge-tree BFS per root, in order; parents[i] / levels[i] receive
        root i's result (int32[n] each, device or host). Host results are copied back while
        the next root is traversed; returns once they are all in place."""
        k = len(roots)
        if len(parents) != k or len(levels) != k:
            raise ValueError("one parent and one level buffer per root")
        ra = (ctypes.c_int64 * max(1, k))(*[int(r) for r in roots])
        pp = (ctypes.c_void_p * max(1, k))(*[_out(x, self.n, "parent") for x in parents])
        lp = (ctypes.c_void_p * max(1, k))(*[_out(x, self.n, "level") for x in levels])
        _check(lib().gt_bfs_roots(self._h, ra, k, pp, lp, _stream(stream)), "gt_bfs_roots")
        return parents, levels

    def bfs_plain(self, root: int, parent=None, level=None, stream=None):
        return self.bfs(root, parent, level, stream, plain=True)

    def autotune(self, nsample: int = 8, seed: int = 1, stream=None) -> gt_tuning:
        """Picks and keeps the fastest gt_tuning for this graph (results never change)."""
        t = gt_tuning()
        _check(lib().gt_autotune(self._h, int(nsample), int(seed), ctypes.byref(t), _stream(stream)), "gt_autotune")
        return t

    def timing(self) -> dict:
        """Phase times (ms) of the last traversal run with time_kernels = 1."""
        t = (ctypes.c_double * 3)()
        _check(lib().gt_bfs_timing(self._h, t), "gt_bfs_timing")
        return {"start_ms": t[0], "loop_ms": t[1], "output_ms": t[2]}

    def trace(self) -> list[dict]:
        cap = 4096
        arr = (gt_level_info * cap)()
        nl = ctypes.c_int32(0)
        _check(lib().gt_bfs_trace(self._h, arr, cap, ctypes.byref(nl)), "gt_bfs_trace")
        out = []
        for i in range(min(nl.value, cap)):
            t = arr[i]
            out.append({"level": t.level, "direction": "bu" if t.direction else "td", "stream": t.direction >= 2,
                        "filtered": t.direction == 3,
                        "frontier": t.frontier,
                        "frontier_edges": t.frontier_edges, "unvisited_edges": t.unvisited_edges,
                        "discovered": t.discovered, "examined": t.examined, "step_ms": t.step_ms})
        return out


def gt_graph_build(edges, n: int, mh: int = 0, keep_plain: bool = True, stream=None, m: int | None = None) -> Graph:
    """Build a graph handle from int64 tuples [m, 2] (numpy/torch host or torch device, or a pointer + m)."""
    if m is None:
        m = _len_pairs(edges)
    cfg = gt_config(mh=int(mh), keep_plain=int(bool(keep_plain)))
    h = ctypes.c_void_p()
    _check(lib().gt_graph_build(_ptr(edges), int(m), int(n), ctypes.byref(cfg), _stream(stream), ctypes.byref(h)),
           "gt_graph_build")
    return Graph(h.value, int(n))


def gt_graph_save(g: Graph, path: str, stream=None) -> None:
    """Write the built graph to `path` (gt_graph_load reads it back)."""
    _check(lib().gt_graph_save(g._h, os.fsencode(path), _stream(stream)), "gt_graph_save")


def gt_graph_load(path: str, stream=None) -> Graph:
    """A graph handle from a file written by gt_graph_save."""
    h = ctypes.c_void_p()
    _check(lib().gt_graph_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "gt_graph_load")
    g = Graph(h.value, 0)
    g.n = int(g.stats()["n"])
    return g


def gt_graph_free(g: Graph):
    g.free()


def gt_graph_stats(g: Graph) -> dict:
    return g.stats()


def gt_graph_vertex_type(g: Graph, out=None, stream=None):
    return g.vertex_type(out, stream)


def gt_graph_degree(g: Graph, out=None, stream=None):
    return g.degree(out, stream)


def gt_graph_set_tuning(g: Graph, t: gt_tuning | None = None, **kw):
    g.set_tuning(t, **kw)


def gt_graph_get_tuning(g: Graph) -> gt_tuning:
    return g.get_tuning()


def gt_bfs(g: Graph, root: int, parent=None, level=None, stream=None):
    return g.bfs(root, parent, level, stream)


def gt_bfs_plain(g: Graph, root: int, parent=None, level=None, stream=None):
    return g.bfs_plain(root, parent, level, stream)


def gt_autotune(g: Graph, nsample: int = 8, seed: int = 1, stream=None) -> gt_tuning:
    return g.autotune(nsample, seed, stream)


def gt_bfs_trace(g: Graph) -> list[dict]:
    return g.trace()


def gt_bfs_batch(graphs, roots_per_graph, parents, levels, stream=None) -> None:
    """Batched BFS: graphs[i] with roots roots_per_graph[i] (a sequence of vertex ids);
    parents[i] / levels[i] are device int32 buffers of len(roots) * n_i (row r = root r)."""
    ng = len(graphs)
    hs = (ctypes.c_void_p * ng)(*[g.handle for g in graphs])
    counts = (ctypes.c_int32 * ng)(*[len(r) for r in roots_per_graph])
    flat = [int(x) for r in roots_per_graph for x in r]
    ra = (ctypes.c_int64 * max(1, len(flat)))(*flat)
    pp = (ctypes.c_void_p * ng)(*[_out(x, len(r) * g.n, "parents") for x, r, g in zip(parents, roots_per_graph, graphs)])
    lp = (ctypes.c_void_p * ng)(*[_out(x, len(r) * g.n, "levels") for x, r, g in zip(levels, roots_per_graph, graphs)])
    _check(lib().gt_bfs_batch(hs, ng, ra, counts, pp, lp, _stream(stream)), "gt_bfs_batch")


class Server:
    """Continuous-batching BFS server over resident graphs (gt_serve_*)."""

    def __init__(self, hbm_budget_bytes: int | None = None, streams: int | None = None,
                 max_batch_roots: int | None = None, window_us: float | None = None,
                 policy: int | None = None, join_levels: int | None = None):
        cfg = gt_serve_config()
        lib().gt_serve_config_default(ctypes.byref(cfg))
        if hbm_budget_bytes is not None:
            cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        if streams is not None:
            cfg.streams = int(streams)
        if max_batch_roots is not None:
            cfg.max_batch_roots = int(max_batch_roots)
        if window_us is not None:
            cfg.window_us = float(window_us)
        if policy is not None:
            cfg.policy = int(policy)
        if join_levels is not None:
            cfg.join_levels = int(join_levels)
        h = ctypes.c_void_p()
        _check(lib().gt_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "gt_serve_create")
        self._h = h.value
        self._graphs = []

    def add_graph(self, g: Graph) -> int:
        gid = ctypes.c_int32(0)
        _check(lib().gt_serve_add_graph(self._h, g.handle, ctypes.byref(gid)), "gt_serve_add_graph")
        self._graphs.append(g)  # keep the handle alive while the server holds it
        return gid.value

    def submit(self, gid: int, root: int, parent, level) -> int:
        t = ctypes.c_uint64(0)
        n = self._graphs[gid].n if 0 <= gid < len(self._graphs) else 0
        _check(lib().gt_serve_submit(self._h, int(gid), int(root), _out(parent, n, "parent"), _out(level, n, "level"),
                                     ctypes.byref(t)), "gt_serve_submit")
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 10000) -> int:
        """0 when done; GT_ETIMEOUT if not yet; raises on failure."""
        rc = lib().gt_serve_poll(self._h, int(ticket), int(timeout_ms))
        if rc not in (GT_OK, GT_ETIMEOUT):
            _check(rc, "gt_serve_poll")
        return rc

    def stats(self) -> dict:
        st = gt_serve_stats()
        _check(lib().gt_serve_get_stats(self._h, ctypes.byref(st)), "gt_serve_get_stats")
        return {k: getattr(st, k) for k, _ in gt_serve_stats._fields_}

    def reset_stats(self):
        _check(lib().gt_serve_reset_stats(self._h), "gt_serve_reset_stats")

    def destroy(self):
        if self._h:
            lib().gt_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def gt_bfs_batch_work(g) -> dict:
    """Work counts of the last gt_bfs_batch call led by graph g (see gt.h)."""
    arr = (ctypes.c_int64 * 4)()
    _check(lib().gt_bfs_batch_work(g._h, arr), "gt_bfs_batch_work")
    return {"pull_entries": arr[0], "push_entries": arr[1], "pull_vertices": arr[2], "discovered": arr[3]}


def gt_test_fail_alloc(after: int = -1) -> None:
    """Allocation-failure injection for tests: the device allocation of graph construction
    after `after` more successful ones fails (GT_ENOMEM); -1 disables it."""
    lib().gt_test_fail_alloc(int(after))


def gt_test_batch_barrier(polls: int = 0, extra: int = 0) -> None:
    """Bounds of the grid-barrier waits of later batched launches (failure tests): with
    extra > 0 every barrier waits for arrivals that never come and gives up after `polls`
    polls, so the launch returns GT_ETIMEOUT. (0, 0) restores the default."""
    lib().gt_test_batch_barrier(int(polls), int(extra))


def gt_bfs_csr_noalloc(row, col, n: int, root: int, parent, level, stream=None) -> None:
    """Plain BFS on a caller's device CSR without any device allocation (fixed scratch;
    n <= 262,144); same results as gt_bfs_plain. row: int64[n + 1], col: int32[row[n]]
    (tensors are checked for dtype, contiguity and length before the call; the length of
    col against row[n] costs one 8-byte read of row)."""
    n = int(n)
    rp = _buf(row, n + 1, "row", "int64")
    cp = _buf(col, 0, "col", "int32")
    if hasattr(row, "numel") and hasattr(col, "numel") and 0 < n < row.numel():
        nnz = int(row[n].item())
        if nnz < 0 or col.numel() < nnz:
            raise ValueError(f"col: row[n] = {nnz} entries, but col holds {col.numel()}")
    _check(lib().gt_bfs_csr_noalloc(rp, cp, n, int(root), _out(parent, n, "parent"),
                                    _out(level, n, "level"), _stream(stream)), "gt_bfs_csr_noalloc")


def gt_count_traversed(edges, level, stream=None, m: int | None = None) -> int:
    """Tuples (device int64 [m, 2]) with both ends reached (device int32 level)."""
    if m is None:
        m = _len_pairs(edges)
    out = ctypes.c_int64(0)
    n = int(level.numel() if hasattr(level, "numel") else len(level))
    _check(lib().gt_count_traversed(_ptr(edges), int(m), _ptr(level), n, ctypes.byref(out), _stream(stream)),
           "gt_count_traversed")
    return int(out.value)

"""Shared test helpers: oracle runs over many roots, and a size-independent BFS certificate."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def oracle_many(og, roots, threads: int | None = None):
    """Oracle (level, parent) for each root; the C oracle releases the GIL, so threads run roots in parallel."""
    threads = threads or min(len(roots), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        return list(ex.map(og.bfs, [int(r) for r in roots]))


def bfs_certificate(edges, level, parent, root: int):
    """Checks, with torch ops on the tuples alone, that (level, parent) is THE BFS answer:
    level[root] = 0 and parent[root] = root; every tuple joins two reached or two unreached
    vertices whose levels differ by <= 1; every other reached v has parent[v] equal to the
    smallest tuple neighbour u with level[u] = level[v] - 1 (which also proves level[v] is
    the hop distance); unreached vertices have parent -1. Works at any size the device holds.
    """
    import torch
    lv = level.long()
    pa = parent.long()
    n = lv.numel()
    assert int(lv[root]) == 0 and int(pa[root]) == root
    u = edges[:, 0]
    v = edges[:, 1]
    keep = u != v
    u, v = u[keep], v[keep]
    lu, lvv = lv[u], lv[v]
    assert bool(((lu >= 0) == (lvv >= 0)).all()), "tuple joins reached and unreached vertices"
    both = (lu >= 0) & (lvv >= 0)
    assert bool(((lu[both] - lvv[both]).abs() <= 1).all()), "levels across a tuple differ by more than 1"
    big = torch.iinfo(torch.int64).max
    best = torch.full((n,), big, dtype=torch.int64, device=lv.device)
    m1 = both & (lu == lvv - 1)   # u one level above v
    best.scatter_reduce_(0, v[m1], u[m1], reduce="amin")
    m2 = both & (lvv == lu - 1)   # v one level above u
    best.scatter_reduce_(0, u[m2], v[m2], reduce="amin")
    reached = lv >= 0
    reached[root] = False
    assert bool((best[reached] != big).all()), "a reached vertex has no neighbour one level up"
    assert bool((pa[reached] == best[reached]).all()), "parent is not the smallest neighbour one level up"
    assert bool((pa[lv < 0] == -1).all()), "unreached vertex with a parent"
    return int((lv >= 0).sum())

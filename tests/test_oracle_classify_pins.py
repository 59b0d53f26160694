"""Pins of the oracle's Alg. 8 (edge-tree vertex classification, Sec. 4.3).

- Hand-derived classes of small graphs at several MH (worked by hand from Alg. 8's
  steps; the path case separates the Jacobi copy of vertex_num_pre from an in-place
  update, which would peel the whole path in one height).
- Structural properties of the edge-tree view (Sec. 4.4): no tree vertex touches a CI
  vertex (property 4); each tree component hangs off at most one core vertex by one
  edge (property 3); tree vertices induce a forest (property 5).
- Identities of Table 2: TL and VZ do not depend on MH, CI+CE+TI is constant, each
  row totals 2^26, and the core shrinks as MH grows.
"""
import os

import numpy as np
import pytest

import graphgen
from oracle import CORE_EDGE, CORE_INTERNAL, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO, OracleGraph

CI, CE, TI, TL, VZ = CORE_INTERNAL, CORE_EDGE, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO
HERE = os.path.dirname(os.path.abspath(__file__))


def classes(pairs, n, mh):
    vt, ph, h = OracleGraph(pairs, n).classify(mh)
    return vt.tolist(), ph.tolist(), h


PATH7 = [(i, i + 1) for i in range(6)]


@pytest.mark.parametrize("mh,expect,height", [
    (0, [TL, CE, CI, CI, CI, CE, TL], 0),
    (1, [TL, TI, CE, CI, CE, TI, TL], 1),
    (2, [TL, TI, TI, CE, TI, TI, TL], 2),
    (3, [TL, TI, TI, TI, TI, TI, TL], 3),
    (-1, [TL, TI, TI, TI, TI, TI, TL], 3),
])
def test_path7(mh, expect, height):
    vt, ph, h = classes(PATH7, 7, mh)
    assert vt == expect and h == height


def test_path7_peel_heights():
    _, ph, _ = classes(PATH7, 7, -1)
    assert ph == [0, 1, 2, 3, 2, 1, 0]


def test_star():
    pairs = [(0, v) for v in range(1, 6)]
    assert classes(pairs, 6, 0)[0] == [CE] + [TL] * 5
    for mh in (1, 2, -1):
        vt, ph, h = classes(pairs, 6, mh)
        assert vt == [TI] + [TL] * 5 and ph[0] == 1 and h == 1


def test_cycle_is_all_core():
    pairs = [(i, (i + 1) % 6) for i in range(6)]
    for mh in (0, 1, -1):
        assert classes(pairs, 6, mh)[0] == [CI] * 6


def test_cycle_with_pendant_path():
    # 4-cycle 0-1-2-3, path 0-4-5 hanging off vertex 0
    pairs = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5)]
    assert classes(pairs, 6, 0)[0] == [CI, CI, CI, CI, CE, TL]
    assert classes(pairs, 6, 1)[0] == [CE, CI, CI, CI, TI, TL]
    vt, _, h = classes(pairs, 6, -1)
    assert vt == [CE, CI, CI, CI, TI, TL] and h == 1


def test_k2_isolated_selfloop_duplicates():
    # 0 isolated, 1-2 a K2 (listed twice), 3 has only a self-loop: degree 0 after cleanup
    pairs = [(1, 2), (2, 1), (3, 3)]
    for mh in (0, 1, -1):
        assert classes(pairs, 4, mh)[0] == [VZ, TL, TL, VZ]


def test_triangle_with_leaves():
    pairs = [(0, 1), (1, 2), (2, 0), (0, 3), (0, 4), (1, 5)]
    assert classes(pairs, 6, 0)[0] == [CE, CE, CI, TL, TL, TL]
    assert classes(pairs, 6, -1)[0] == [CE, CE, CI, TL, TL, TL]


def test_spider():
    # centre 0 with legs 0-1-2, 0-3-4 and 0-5
    pairs = [(0, 1), (1, 2), (0, 3), (3, 4), (0, 5)]
    assert classes(pairs, 6, 0)[0] == [CE, CE, TL, CE, TL, TL]
    assert classes(pairs, 6, 1)[0] == [CE, TI, TL, TI, TL, TL]
    vt, ph, h = classes(pairs, 6, 2)
    assert vt == [TI, TI, TL, TI, TL, TL] and h == 2 and ph[0] == 2


def tree_structure_checks(row, col, vt):
    n = row.shape[0] - 1
    deg = np.diff(row)
    src = np.repeat(np.arange(n), deg)
    is_tree = (vt == TI) | (vt == TL)
    is_core = (vt == CI) | (vt == CE)
    assert ((vt == VZ) == (deg == 0)).all()
    assert ((vt == TL) == (deg == 1)).all()
    # property 4: no tree vertex is adjacent to a CI vertex
    assert not (is_tree[src] & (vt[col] == CI)).any()
    # CE = core vertices with at least one tree neighbour
    has_tree_nb = np.zeros(n, dtype=bool)
    np.logical_or.at(has_tree_nb, src[is_tree[col]], True)
    assert ((vt == CE) == (is_core & has_tree_nb)).all()
    # properties 3 and 5 by union-find over tree-tree edges
    parent = np.arange(n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    tt = is_tree[src] & is_tree[col] & (src < col)
    n_tt = int(tt.sum())
    for a, b in zip(src[tt].tolist(), col[tt].tolist()):
        ra, rb = find(a), find(b)
        assert ra != rb, "tree vertices contain a cycle"
        parent[ra] = rb
    comps = {find(v) for v in np.flatnonzero(is_tree).tolist()}
    assert n_tt == int(is_tree.sum()) - len(comps)  # a forest
    attach = {}
    tc = is_tree[src] & is_core[col]
    for a, c in zip(src[tc].tolist(), col[tc].tolist()):
        attach.setdefault(find(a), []).append((a, c))
    assert all(len(v) == 1 for v in attach.values()), "a tree hangs off the core by more than one edge"


@pytest.mark.parametrize("scale", [10, 12])
def test_rmat_structure_and_table2_identities(scale):
    n = 1 << scale
    e = graphgen.rmat_edges(scale, 16, seed=5 + scale)
    g = OracleGraph(e, n)
    row, col = g.csr()
    counts = {}
    core_prev = None
    for mh in (0, 1, 2, -1):
        vt, ph, h = g.classify(mh)
        tree_structure_checks(row, col, vt)
        assert mh == -1 or h <= mh
        assert ph.max() <= (h if mh == -1 else mh)
        c = np.bincount(vt, minlength=5)
        assert c.sum() == n
        counts[mh] = c
        core = (vt == CI) | (vt == CE)
        if core_prev is not None:
            assert not (core & ~core_prev).any(), "the core must shrink as MH grows"
        core_prev = core
    for mh in (1, 2, -1):
        assert counts[mh][TL] == counts[0][TL] and counts[mh][VZ] == counts[0][VZ]
        assert counts[mh][CI] + counts[mh][CE] + counts[mh][TI] == counts[0][CI] + counts[0][CE]
    assert counts[0][TI] == 0


def test_table2_fixture_identities():
    rows = [list(map(int, ln.split())) for ln in open(os.path.join(HERE, "golden", "table2_s26_classes.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert [r[0] for r in rows] == [0, 1, 2]
    for r in rows:
        assert sum(r[1:]) == 1 << 26
        assert r[4] == rows[0][4] and r[5] == rows[0][5]
        assert r[1] + r[2] + r[3] == rows[0][1] + rows[0][2]
    assert rows[0][3] == 0
    # VZ and TL shares quoted in Sec. 4.1: 51.1 % and 12.4 %
    assert round(100 * rows[0][5] / (1 << 26), 1) == 51.1
    assert round(100 * rows[0][4] / (1 << 26), 1) == 12.4

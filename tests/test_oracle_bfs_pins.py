"""Pins of the CPU oracle's CSR build and BFS against facts that do not come from the oracle.

- Exhaustive brute force: every simple graph on <= 5 vertices (and random ones on 6-7),
  levels from Floyd-Warshall all-pairs distances (a different algorithm from the oracle's
  queue), parents from the literal min-id definition scanned over all vertices.
- Closed forms: path, cycle, star, complete graph, grid, complete binary tree, K2,
  disconnected pieces, isolated root.
- BFS invariants on R-MAT graphs: level[root] = 0, levels across an edge differ by <= 1,
  every parent is a neighbour one level up and the smallest such.
- CSR against a set-of-pairs construction with duplicates and self-loops planted.
- TEPS numerator (traversed_tuples) against counts fixed by hand on a tuple list with
  duplicates, self-loops on reached and unreached vertices and a second component.
  Checked by hand: skipping self-loops, testing level > 0, or stopping one tuple early in
  or_traversed_tuples each fails these tests.
"""
import itertools

import numpy as np
import pytest

import graphgen
from oracle import OracleGraph, traversed_tuples


def noisy_tuples(pairs, n, rng):
    """Tuples of the edge set `pairs` with random duplicates, flipped ends and self-loops."""
    out = []
    for (a, b) in pairs:
        for _ in range(int(rng.integers(1, 3))):
            out.append((a, b) if rng.random() < 0.5 else (b, a))
    for _ in range(int(rng.integers(0, 3))):
        v = int(rng.integers(0, n))
        out.append((v, v))
    rng.shuffle(out)
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def brute_force(n, pairs, root):
    inf = 10 ** 9
    d = np.full((n, n), inf, dtype=np.int64)
    np.fill_diagonal(d, 0)
    adj = [[False] * n for _ in range(n)]
    for a, b in pairs:
        if a != b:
            d[a, b] = d[b, a] = 1
            adj[a][b] = adj[b][a] = True
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    level = np.where(d[root] >= inf, -1, d[root]).astype(np.int32)
    parent = np.full(n, -1, dtype=np.int32)
    parent[root] = root
    for v in range(n):
        if v == root or level[v] < 0:
            continue
        cands = [u for u in range(n) if adj[u][v] and level[u] == level[v] - 1]
        parent[v] = min(cands)
    return level, parent


def check_against_brute(n, pairs, rng):
    tuples = noisy_tuples(pairs, n, rng) if pairs else np.zeros((0, 2), dtype=np.int64)
    g = OracleGraph(tuples, n)
    for root in range(n):
        lv, pa = g.bfs(root)
        blv, bpa = brute_force(n, pairs, root)
        assert np.array_equal(lv, blv), (n, pairs, root)
        assert np.array_equal(pa, bpa), (n, pairs, root)


def test_exhaustive_small_graphs():
    rng = np.random.default_rng(7)
    for n in range(1, 6):
        all_pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(all_pairs)):
            pairs = [p for i, p in enumerate(all_pairs) if mask >> i & 1]
            check_against_brute(n, pairs, rng)


@pytest.mark.parametrize("n", [6, 7])
def test_random_graphs_6_7(n):
    rng = np.random.default_rng(100 + n)
    all_pairs = list(itertools.combinations(range(n), 2))
    for _ in range(300):
        keep = rng.random(len(all_pairs)) < rng.uniform(0.1, 0.7)
        pairs = [p for p, k in zip(all_pairs, keep) if k]
        check_against_brute(n, pairs, rng)


def test_path_closed_form():
    n = 50
    g = OracleGraph([(i, i + 1) for i in range(n - 1)], n)
    lv, pa = g.bfs(0)
    assert lv.tolist() == list(range(n))
    assert pa.tolist() == [0] + list(range(n - 1))
    r = 20
    lv, pa = g.bfs(r)
    assert lv.tolist() == [abs(i - r) for i in range(n)]
    assert pa.tolist() == [i + 1 if i < r else (r if i == r else i - 1) for i in range(n)]


@pytest.mark.parametrize("n", [7, 8, 33])
def test_cycle_closed_form(n):
    g = OracleGraph([(i, (i + 1) % n) for i in range(n)], n)
    lv, pa = g.bfs(0)
    assert lv.tolist() == [min(i, n - i) for i in range(n)]
    exp = [0]
    for i in range(1, n):
        if 2 * i < n:
            exp.append(i - 1)
        elif 2 * i > n:
            exp.append((i + 1) % n)
        else:  # antipode of an even cycle: both neighbours one level up, smaller wins
            exp.append(min(i - 1, (i + 1) % n))
    assert pa.tolist() == exp


def test_star_complete_k2_isolated():
    k = 9  # star: centre 4, leaves the rest
    g = OracleGraph([(4, v) for v in range(k) if v != 4], k)
    lv, pa = g.bfs(7)
    assert lv[7] == 0 and lv[4] == 1 and pa[4] == 7
    assert all(lv[v] == 2 and pa[v] == 4 for v in range(k) if v not in (4, 7))
    n = 12
    g = OracleGraph(list(itertools.combinations(range(n), 2)), n)
    lv, pa = g.bfs(5)
    assert lv.tolist() == [0 if v == 5 else 1 for v in range(n)]
    assert pa.tolist() == [5] * n
    g = OracleGraph([(3, 1)], 4)  # K2 plus two isolated vertices
    lv, pa = g.bfs(3)
    assert lv.tolist() == [-1, 1, -1, 0] and pa.tolist() == [-1, 3, -1, 3]
    lv, pa = g.bfs(0)  # isolated root
    assert lv.tolist() == [0, -1, -1, -1] and pa.tolist() == [0, -1, -1, -1]


def test_grid_closed_form():
    a, b = 9, 13
    pairs = [(x * b + y, x * b + y + 1) for x in range(a) for y in range(b - 1)]
    pairs += [(x * b + y, (x + 1) * b + y) for x in range(a - 1) for y in range(b)]
    g = OracleGraph(pairs, a * b)
    lv, pa = g.bfs(0)
    for x in range(a):
        for y in range(b):
            v = x * b + y
            assert lv[v] == x + y
            if v:
                assert pa[v] == ((x - 1) * b + y if x > 0 else v - 1)


def test_binary_tree_and_components():
    n = 127
    pairs = [(i, (i - 1) // 2) for i in range(1, n)]
    pairs += [(n + i, n + i + 1) for i in range(9)]  # a second component: path on 10 vertices
    g = OracleGraph(pairs, n + 10)
    lv, pa = g.bfs(0)
    for i in range(n):
        assert lv[i] == int(np.floor(np.log2(i + 1)))
        assert pa[i] == (0 if i == 0 else (i - 1) // 2)
    assert (lv[n:] == -1).all() and (pa[n:] == -1).all()


def test_csr_against_sets():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = int(rng.integers(1, 60))
        m = int(rng.integers(0, 200))
        t = rng.integers(0, n, size=(m, 2)).astype(np.int64)
        g = OracleGraph(t, n)
        row, col = g.csr()
        nbrs = [set() for _ in range(n)]
        for a, b in t.tolist():
            if a != b:
                nbrs[a].add(b)
                nbrs[b].add(a)
        assert row[0] == 0 and row.shape == (n + 1,)
        for v in range(n):
            assert col[row[v]:row[v + 1]].tolist() == sorted(nbrs[v])
        assert g.nnz == sum(len(s) for s in nbrs)


def test_bad_ids_rejected():
    with pytest.raises(ValueError):
        OracleGraph([(0, 5)], 5)
    with pytest.raises(ValueError):
        OracleGraph([(-1, 0)], 5)


def check_invariants(row, col, root, lv, pa):
    n = row.shape[0] - 1
    assert lv[root] == 0 and pa[root] == root
    src = np.repeat(np.arange(n), np.diff(row))
    a, b = lv[src], lv[col]
    both = (a >= 0) & (b >= 0)
    assert ((a >= 0) == (b >= 0)).all(), "an edge joins a reached and an unreached vertex"
    assert (np.abs(a[both] - b[both]) <= 1).all()
    reached = np.flatnonzero(lv >= 0)
    assert ((pa >= 0) == (lv >= 0)).all()
    for v in reached.tolist():
        if v == root:
            continue
        nb = col[row[v]:row[v + 1]]
        up = nb[lv[nb] == lv[v] - 1]
        assert up.size > 0 and pa[v] == up.min()


@pytest.mark.parametrize("scale", [8, 10, 12])
def test_rmat_invariants(scale):
    e = graphgen.rmat_edges(scale, 16, seed=scale)
    n = 1 << scale
    g = OracleGraph(e, n)
    row, col = g.csr()
    roots = graphgen.pick_roots(11, n, 4, np.diff(row))
    for r in roots.tolist():
        lv, pa = g.bfs(r)
        check_invariants(row, col, r, lv, pa)
        # the TEPS numerator counts the tuples inside the root's component
        cnt = traversed_tuples(e, lv)
        assert cnt == int(((lv[e[:, 0]] >= 0) & (lv[e[:, 1]] >= 0)).sum())


# Hand-built tuple list for the TEPS numerator (Graph500 convention, Sec. 6.1: every input
# tuple whose two ends are reached counts once, duplicates and self-loops included).
HAND_TUPLES = [
    (0, 1),  # 0
    (1, 0),  # 1  duplicate of 0, ends flipped
    (1, 2),  # 2
    (2, 2),  # 3  self-loop on a vertex reached from 0
    (0, 1),  # 4  duplicate of 0, same order
    (3, 4),  # 5  second component
    (5, 5),  # 6  self-loop on a vertex with no other edge
    (4, 4),  # 7  self-loop in the second component
    (2, 0),  # 8
    (6, 3),  # 9  second component, last tuple
]


@pytest.mark.parametrize("root,want", [(0, 6), (1, 6), (3, 3), (6, 3), (5, 1)])
def test_traversed_tuples_hand_counts(root, want):
    """Counts fixed by hand from the list above: root 0 or 1 reaches {0, 1, 2} (tuples 0-4
    and 8: the two duplicates and the self-loop count); root 3 or 6 reaches {3, 4, 6}
    (tuples 5, 7, 9); root 5 reaches only itself, and its self-loop counts. Dropping
    self-loops, merging duplicates, skipping the root (level 0) or the last tuple each
    change one of these numbers."""
    e = np.array(HAND_TUPLES, dtype=np.int64)
    g = OracleGraph(e, 7)
    lv, _ = g.bfs(root)
    assert traversed_tuples(e, lv) == want


def test_traversed_tuples_given_levels():
    """The count depends only on which ends have level >= 0, whatever the levels are."""
    e = np.array(HAND_TUPLES, dtype=np.int64)
    assert traversed_tuples(e, np.full(7, -1, np.int32)) == 0
    assert traversed_tuples(e, np.array([-1, -1, 7, -1, -1, -1, -1], np.int32)) == 1   # tuple 3
    assert traversed_tuples(e, np.array([-1, -1, -1, 0, 2, -1, -1], np.int32)) == 2    # tuples 5, 7
    assert traversed_tuples(e, np.array([-1, -1, -1, -1, -1, -1, 0], np.int32)) == 0   # 6's tuple needs 3
    assert traversed_tuples(e, np.zeros(7, np.int32)) == 10

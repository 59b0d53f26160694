"""Batched BFS (64-root lane words, one persistent launch) through the C-ABI: every row
must equal the single-root answer bit for bit (checked against the CPU oracle)."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from helpers import oracle_many
from oracle import OracleGraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def run_batch(torch, graphs, roots):
    outs_p, outs_l = [], []
    for g, r in zip(graphs, roots):
        outs_p.append(torch.full((max(len(r), 1), g.n), -7, dtype=torch.int32, device="cuda"))
        outs_l.append(torch.full((max(len(r), 1), g.n), -7, dtype=torch.int32, device="cuda"))
    gt.gt_bfs_batch(graphs, roots, outs_p, outs_l)
    torch.cuda.synchronize()
    return [p.cpu().numpy() for p in outs_p], [l.cpu().numpy() for l in outs_l]


def check_rows(P, L, og, roots, what):
    want = oracle_many(og, roots)
    for i, (r, (wl, wp)) in enumerate(zip(roots, want)):
        if not np.array_equal(L[i], wl):
            bad = np.flatnonzero(L[i] != wl)[:8]
            raise AssertionError(f"{what} root {r}: level differs at {bad.tolist()}: {L[i][bad]} vs {wl[bad]}")
        if not np.array_equal(P[i], wp):
            bad = np.flatnonzero(P[i] != wp)[:8]
            raise AssertionError(f"{what} root {r}: parent differs at {bad.tolist()}: {P[i][bad]} vs {wp[bad]}")


def test_batch_one_word_scale16(torch):
    n = 1 << 16
    e = graphgen.rmat_edges(16, 16, seed=1)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(2, n, 64, og.degree()).tolist()
    (P,), (L,) = run_batch(torch, [g], [roots])
    check_rows(P, L, og, roots, "s16 batch")


def test_batch_partial_second_word_and_duplicates(torch):
    n = 1 << 14
    e = graphgen.rmat_edges(14, 16, seed=3)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(4, n, 90, og.degree()).tolist()
    roots += roots[:7]  # the same root in several lanes
    (P,), (L,) = run_batch(torch, [g], [roots])
    check_rows(P, L, og, roots, "s14 97 roots")


@pytest.mark.parametrize("mh", [0, 1, -1])
def test_batch_every_root_class(torch, mh):
    n = 1 << 13
    e = graphgen.rmat_edges(13, 8, seed=11)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n, mh=mh)
    vt = g.vertex_type()
    rng = np.random.default_rng(5)
    roots = []
    for cls in range(5):
        ids = np.flatnonzero(vt == cls)
        if ids.size:
            roots += rng.choice(ids, size=min(15, ids.size), replace=False).tolist()
    (P,), (L,) = run_batch(torch, [g], [roots])
    check_rows(P, L, og, roots, f"mh={mh}")


def test_batch_mixed_graphs(torch):
    specs = [("rmat", 10, None), ("rmat", 12, None), ("uniform", 20000, 16), ("rmat", 15, None), ("rmat", 11, None)]
    graphs, oracles, roots = [], [], []
    for i, (kind, a, d) in enumerate(specs):
        if kind == "rmat":
            n = 1 << a
            e = graphgen.rmat_edges(a, 16, seed=30 + i)
        else:
            n = a
            e = graphgen.uniform_edges(n, n * d // 2, seed=30 + i)
        og = OracleGraph(e, n)
        graphs.append(gt.gt_graph_build(e, n))
        oracles.append(og)
        k = [64, 20, 64, 130, 0][i]
        roots.append(graphgen.pick_roots(40 + i, n, k, og.degree()).tolist() if k else [])
    P, L = run_batch(torch, graphs, roots)
    for i, og in enumerate(oracles):
        if roots[i]:
            check_rows(P[i], L[i], og, roots[i], f"mixed graph {i}")


HAND = {
    "k2_and_isolated": ([(2, 3), (5, 6), (6, 5)], 8),
    "spider": ([(0, 1), (1, 2), (0, 3), (3, 4), (0, 5), (5, 6), (6, 7)], 8),
    "path": ([(i, i + 1) for i in range(20)], 21),
    "lollipop": ([(i, (i + 1) % 6) for i in range(6)] + [(5, 6), (6, 7), (7, 8), (8, 9), (7, 10)], 11),
}


@pytest.mark.parametrize("mh", [0, 2, -1])
def test_batch_hand_graphs_all_roots(torch, mh):
    graphs, oracles, roots = [], [], []
    for name, (pairs, n) in sorted(HAND.items()):
        e = np.array(pairs, dtype=np.int64)
        oracles.append(OracleGraph(e, n))
        graphs.append(gt.gt_graph_build(e, n, mh=mh))
        roots.append(list(range(n)))
    P, L = run_batch(torch, graphs, roots)
    for i, og in enumerate(oracles):
        check_rows(P[i], L[i], og, roots[i], f"hand {i} mh={mh}")


def test_batch_equals_single_calls_and_repeats(torch):
    n = 1 << 15
    e = graphgen.rmat_edges(15, 16, seed=8)
    g = gt.gt_graph_build(e, n)
    deg = g.degree()
    roots = graphgen.pick_roots(9, n, 64, deg).tolist()
    for rep in range(2):  # second call reuses the slot storage
        (P,), (L,) = run_batch(torch, [g], [roots])
        for i, r in enumerate(roots[:16]):
            p, l = g.bfs(r)
            assert np.array_equal(L[i], l) and np.array_equal(P[i], p), f"rep {rep} root {r}"


@pytest.mark.parametrize("batch_alpha", [1, 14, 1 << 30])
def test_batch_hubs_span_several_chunks(torch, batch_alpha):
    # four hubs of degree ~5000 (adjacencies cut into several work chunks, so parents are
    # merged across chunks) over a sparse random graph; both directions forced in turn
    rng = np.random.default_rng(31)
    n = 12000
    pairs = [graphgen.uniform_edges(n, 3 * n, seed=32)]
    for h in range(4):
        nb = rng.choice(np.arange(4, n), size=5000, replace=False)
        pairs.append(np.stack([np.full(nb.size, h), nb], axis=1))
    e = np.concatenate(pairs).astype(np.int64)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    g.set_tuning(batch_alpha=batch_alpha)
    roots = [0, 1, 2, 3] + graphgen.pick_roots(33, n, 60, og.degree()).tolist()
    (P,), (L,) = run_batch(torch, [g], [roots])
    check_rows(P, L, og, roots, f"hubs alpha={batch_alpha}")


def test_batch_graph_replay_takes_new_roots_and_outputs(torch):
    # the batched launch is a captured graph replayed while its shape is unchanged: a second
    # call with other roots and other output buffers must use them; a call with another
    # shape (more lane words) recaptures
    n = 1 << 14
    e = graphgen.rmat_edges(14, 16, seed=21)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    cand = graphgen.pick_roots(22, n, 200, og.degree()).tolist()
    for roots in (cand[:64], cand[64:128], cand[:150], cand[150:200]):
        (P,), (L,) = run_batch(torch, [g], [roots])
        check_rows(P, L, og, roots, f"replay {len(roots)} roots")


def test_batch_rejects_too_many_lane_words(torch):
    n = 1 << 10
    e = graphgen.rmat_edges(10, 16, seed=23)
    g = gt.gt_graph_build(e, n)
    roots = [0] * (64 * 256 + 1)  # one lane word more than one launch takes
    p = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GtError) as ei:
        gt.gt_bfs_batch([g], [roots], [p], [p])
    assert ei.value.code == gt.GT_EINVAL


def test_batch_same_graph_twice(torch):
    # one handle listed twice takes separate lane-word storage for each list
    n = 1 << 13
    e = graphgen.rmat_edges(13, 16, seed=25)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    cand = graphgen.pick_roots(26, n, 100, og.degree()).tolist()
    r1, r2 = cand[:70], cand[70:]
    P, L = run_batch(torch, [g, g], [r1, r2])
    check_rows(P[0], L[0], og, r1, "first list")
    check_rows(P[1], L[1], og, r2, "second list")


def test_batch_work_counts(torch):
    """The launch's work counts (the batched roofline's inputs): with one root in the lane
    word every reached core vertex but the start is discovered exactly once; with 64 roots
    the pull and push phases both read adjacency entries."""
    n = 1 << 14
    e = graphgen.rmat_edges(14, 16, seed=27)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    core = np.isin(g.vertex_type(), [0, 1])  # CI, CE
    deg = og.degree()
    r = int(np.flatnonzero(core & (deg > 2))[0])
    (P,), (L,) = run_batch(torch, [g], [[r]])
    lv = L[0]
    w = gt.gt_bfs_batch_work(g)
    assert w["discovered"] == int((core & (lv >= 0)).sum()) - 1
    roots = graphgen.pick_roots(28, n, 64, deg).tolist()
    run_batch(torch, [g], [roots])
    w = gt.gt_bfs_batch_work(g)
    assert w["pull_entries"] > 0 and w["push_entries"] > 0 and w["pull_vertices"] > 0
    assert w["discovered"] >= int(core.sum() * 0.5)


def test_batch_large_core_medium_rows(torch):
    """R-MAT scale 21: its core (about 966 K vertices) is above the size (2^19) from which
    core vertices of degree 33-128 are scanned 32 to a warp as one flattened sequence, so
    all three work lists (short rows a lane each, medium rows flattened, long rows in
    chunks) take part; every row must equal the oracle."""
    scale = 21
    n = 1 << scale
    e = graphgen.rmat_edges(scale, 16, seed=41)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    assert g.stats()["n_core"] >= 1 << 19
    row, col = og.csr()
    vt = g.vertex_type()
    core = np.isin(vt, [0, 1])
    cdeg = np.bincount(np.repeat(np.arange(n), np.diff(row))[core[col]], minlength=n)[core]
    assert ((cdeg > 32) & (cdeg <= 128)).sum() > 1000  # medium rows present
    roots = graphgen.pick_roots(42, n, 64, og.degree()).tolist()
    (P,), (L,) = run_batch(torch, [g], [roots])
    check_rows(P, L, og, roots, "s21 large core")
    # the same graph beside a small one (no medium list) in one launch: each slot takes
    # its pull work from its own counters
    ns = 1 << 12
    es = graphgen.rmat_edges(12, 16, seed=43)
    ogs = OracleGraph(es, ns)
    gs = gt.gt_graph_build(es, ns)
    rs = graphgen.pick_roots(44, ns, 70, ogs.degree()).tolist()
    P2, L2 = run_batch(torch, [gs, g], [rs, roots[:40]])
    check_rows(P2[0], L2[0], ogs, rs, "small graph beside s21")
    check_rows(P2[1], L2[1], og, roots[:40], "s21 beside small graph")

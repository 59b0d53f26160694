"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, element by element.

Bar: bit-exact for every integer output (CSR degrees, Alg. 8 classes, levels, min-id
parents); there is no floating point on the path.
"""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from helpers import bfs_certificate, oracle_many
from oracle import CORE_EDGE, CORE_INTERNAL, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO, OracleGraph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def build_pair(edges, n, mh=0):
    return OracleGraph(edges, n), gt.gt_graph_build(np.ascontiguousarray(edges, dtype=np.int64), n, mh=mh)


def bfs_dev(torch, g, root, plain=False):
    n = g.n
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    l = torch.empty(n, dtype=torch.int32, device="cuda")
    p.fill_(-7)
    l.fill_(-7)  # garbage the library must overwrite
    g.bfs(int(root), p, l, plain=plain)
    torch.cuda.synchronize()
    return l.cpu().numpy(), p.cpu().numpy()


def assert_same(got, want, what):
    gl, gp = got
    wl, wp = want
    if not np.array_equal(gl, wl):
        bad = np.flatnonzero(gl != wl)[:10]
        raise AssertionError(f"{what}: level differs at {bad.tolist()}: got {gl[bad].tolist()} want {wl[bad].tolist()}")
    if not np.array_equal(gp, wp):
        bad = np.flatnonzero(gp != wp)[:10]
        raise AssertionError(f"{what}: parent differs at {bad.tolist()}: got {gp[bad].tolist()} want {wp[bad].tolist()}")


# ---- inputs and build ------------------------------------------------------------------

def test_device_generator_matches_host(torch_cuda):
    torch = torch_cuda
    for scale in (1, 10, 16):
        m = 16 << scale
        host = graphgen.rmat_edges(scale, 16, seed=21)
        dev = torch.empty((m, 2), dtype=torch.int64, device="cuda")
        graphgen.rmat_edges_device(dev.data_ptr(), scale, m, seed=21)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host)
    host = graphgen.uniform_edges(12345, 99999, seed=3)
    dev = torch.empty((99999, 2), dtype=torch.int64, device="cuda")
    graphgen.uniform_edges_device(dev.data_ptr(), 12345, 99999, seed=3)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)


@pytest.mark.parametrize("scale", [8, 12, 16])
def test_csr_and_classes_parity(torch_cuda, scale):
    n = 1 << scale
    e = graphgen.rmat_edges(scale, 16, seed=100 + scale)
    og = OracleGraph(e, n)
    for mh in (0, 1, 2, -1):
        g = gt.gt_graph_build(e, n, mh=mh)
        assert np.array_equal(g.degree(), og.degree())
        vt_o, _, h_o = og.classify(mh)
        vt_g = g.vertex_type()
        assert np.array_equal(vt_g, vt_o), f"classes differ at mh={mh}"
        st = g.stats()
        cnt = np.bincount(vt_o, minlength=5)
        assert st["nnz"] == og.nnz and st["n_class"] == cnt.tolist() and st["height"] == h_o
        assert st["n_core"] == cnt[CORE_INTERNAL] + cnt[CORE_EDGE]
        g.free()


def test_device_resident_tuples(torch_cuda):
    torch = torch_cuda
    e = graphgen.rmat_edges(12, 16, seed=5)
    n = 1 << 12
    g1 = gt.gt_graph_build(e, n)
    g2 = gt.gt_graph_build(torch.from_numpy(e).cuda(), n)
    assert np.array_equal(g1.vertex_type(), g2.vertex_type())
    assert_same(bfs_dev(torch, g2, 7), bfs_dev(torch, g1, 7), "device tuples")


# ---- BFS parity -------------------------------------------------------------------------

def test_bfs_scale16_config(torch_cuda):
    """Plain single-source BFS, R-MAT scale 16, edge factor 16, 16 seeded roots of degree >= 1."""
    torch = torch_cuda
    scale, n = 16, 1 << 16
    e = graphgen.rmat_edges(scale, 16, seed=1)
    og, g = build_pair(e, n)
    roots = graphgen.pick_roots(2, n, 16, og.degree())
    want = oracle_many(og, roots)
    for r, w in zip(roots.tolist(), want):
        assert_same(bfs_dev(torch, g, r), w, f"edge-tree root {r}")
        assert_same(bfs_dev(torch, g, r, plain=True), w, f"plain root {r}")


@pytest.mark.parametrize("mh", [0, 1, 2, -1])
def test_bfs_every_root_class(torch_cuda, mh):
    torch = torch_cuda
    scale, n = 14, 1 << 14
    e = graphgen.rmat_edges(scale, 8, seed=77)
    og, g = build_pair(e, n, mh)
    vt = g.vertex_type()
    rng = np.random.default_rng(mh + 10)
    roots = []
    for cls in (CORE_INTERNAL, CORE_EDGE, TREE_INTERNAL, TREE_LEAF, VERTEX_ZERO):
        ids = np.flatnonzero(vt == cls)
        if ids.size:
            roots += rng.choice(ids, size=min(4, ids.size), replace=False).tolist()
    want = oracle_many(og, roots)
    for r, w in zip(roots, want):
        assert_same(bfs_dev(torch, g, r), w, f"mh={mh} root {r} class {vt[r]}")


HAND = {
    "path": ([(i, i + 1) for i in range(40)], 41),
    "star": ([(0, i) for i in range(1, 30)], 30),
    "cycle": ([(i, (i + 1) % 25) for i in range(25)], 25),
    "k2_and_isolated": ([(2, 3), (5, 6), (6, 5)], 8),
    "spider": ([(0, 1), (1, 2), (0, 3), (3, 4), (0, 5), (5, 6), (6, 7)], 8),
    "binary_tree": ([(i, (i - 1) // 2) for i in range(1, 63)], 63),
    "lollipop": ([(i, (i + 1) % 6) for i in range(6)] + [(5, 6), (6, 7), (7, 8), (8, 9), (7, 10)], 11),
    "two_components": ([(0, 1), (1, 2), (2, 0), (2, 3), (4, 5), (5, 6), (6, 7), (7, 4), (4, 8)], 9),
    "self_loops_only": ([(0, 0), (1, 1), (2, 2)], 4),
}


@pytest.mark.parametrize("name", sorted(HAND))
@pytest.mark.parametrize("mh", [0, 1, 2, -1])
def test_hand_graphs_all_roots(torch_cuda, name, mh):
    torch = torch_cuda
    pairs, n = HAND[name]
    og, g = build_pair(np.array(pairs, dtype=np.int64), n, mh)
    vt_o, _, _ = og.classify(mh)
    assert np.array_equal(g.vertex_type(), vt_o)
    for r in range(n):
        assert_same(bfs_dev(torch, g, r), og.bfs(r), f"{name} mh={mh} root {r}")
        assert_same(bfs_dev(torch, g, r, plain=True), og.bfs(r), f"{name} plain root {r}")


def test_direction_and_launch_mode_independence(torch_cuda):
    torch = torch_cuda
    scale, n = 15, 1 << 15
    e = graphgen.rmat_edges(scale, 16, seed=9)
    og, g = build_pair(e, n)
    roots = graphgen.pick_roots(5, n, 4, og.degree())
    want = oracle_many(og, roots)
    for force in (0, 1, 2):
        for mode in (0, 1):
            for thr in ((32, 1024, 32768, 8), (1, 2, 3, 0), (8, 16, 64, 1000), (4, 1 << 20, 1 << 30, 2)):
                g.set_tuning(force_direction=force, launch_mode=mode, td_warp_min=thr[0], td_cta_min=thr[1],
                             td_grid_min=thr[2], bu_thread_scan=thr[3], blocks_per_sm=1 + force)
                for r, w in zip(roots.tolist(), want):
                    what = f"force={force} mode={mode} thr={thr} root {r}"
                    assert_same(bfs_dev(torch, g, r), w, what)
                    assert_same(bfs_dev(torch, g, r, plain=True), w, what + " plain")


def test_degree_aware_bottom_up(torch_cuda):
    # Alg. 3 order (highest-degree neighbour first, min-id parents restored after the loop)
    # gives the oracle's levels and parents, with the switch and with bottom-up forced, on
    # the core and plain views, an R-MAT graph and the hand-made graphs (every root)
    torch = torch_cuda
    scale, n = 14, 1 << 14
    e = graphgen.rmat_edges(scale, 16, seed=19)
    og, g = build_pair(e, n)
    roots = graphgen.pick_roots(6, n, 6, og.degree())
    want = oracle_many(og, roots)
    for force in (0, 2):
        g.set_tuning(bu_hub_first=1, force_direction=force)
        for r, w in zip(roots.tolist(), want):
            assert_same(bfs_dev(torch, g, r), w, f"hub force={force} root {r}")
            assert_same(bfs_dev(torch, g, r, plain=True), w, f"hub force={force} plain root {r}")
    g.free()
    for name in sorted(HAND):
        pairs, nh = HAND[name]
        og, g = build_pair(np.array(pairs, dtype=np.int64), nh, 0)
        g.set_tuning(bu_hub_first=1, force_direction=2)
        for r in range(nh):
            assert_same(bfs_dev(torch, g, r), og.bfs(r), f"hub {name} root {r}")
            assert_same(bfs_dev(torch, g, r, plain=True), og.bfs(r), f"hub {name} plain root {r}")
        g.free()


def test_trace_directions(torch_cuda):
    torch = torch_cuda
    n = 1 << 16
    e = graphgen.rmat_edges(16, 16, seed=1)
    g = gt.gt_graph_build(e, n)
    r = int(graphgen.pick_roots(2, n, 1, g.degree())[0])
    g.set_tuning(count_work=1)
    bfs_dev(torch, g, r)
    tr = g.trace()
    assert tr and tr[0]["frontier"] == 1
    assert {t["direction"] for t in tr} == {"td", "bu"}  # the switch does fire on R-MAT
    # bottom-up levels stream over all vertices while most are unvisited, then scan the
    # gathered list (both forms are in every oracle comparison of this module)
    bu = [t for t in tr if t["direction"] == "bu"]
    assert bu[0]["stream"] and not bu[-1]["stream"]
    assert all(t["examined"] >= 0 for t in tr)
    # plain BFS on the whole graph: every reached vertex but the root is discovered on
    # exactly one traced level, and the loop stops once no unvisited edge is left
    lv, _ = bfs_dev(torch, g, r, plain=True)
    tp = g.trace()
    assert sum(t["discovered"] for t in tp) + 1 == int((lv >= 0).sum())
    assert all(t["unvisited_edges"] > 0 for t in tp[1:])
    g.set_tuning(force_direction=1)
    bfs_dev(torch, g, r)
    assert {t["direction"] for t in g.trace()} == {"td"}


def test_filtered_bottom_up_levels(torch_cuda):
    """Roots whose first bottom-up level follows a top-down level with a small frontier run
    the filtered streaming step (trace direction 3); their answers equal the oracle's, and so
    do the same roots with the filter never taken (all bottom-up from the start)."""
    torch = torch_cuda
    n = 1 << 18
    e = graphgen.rmat_edges(18, 16, seed=41)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(42, n, 24, og.degree()).tolist()
    want = oracle_many(og, roots)
    filtered = 0
    for r, w in zip(roots, want):
        for plain in (False, True):
            assert_same(bfs_dev(torch, g, r, plain), w, f"root {r} plain={plain}")
            filtered += any(t["filtered"] for t in g.trace())
    assert filtered > 0, "no traversal took the filtered bottom-up step"
    g.set_tuning(force_direction=2)
    for r, w in zip(roots[:6], want[:6]):
        assert_same(bfs_dev(torch, g, r), w, f"all bottom-up root {r}")
        assert not any(t["filtered"] for t in g.trace())


def test_host_output_buffers(torch_cuda):
    torch = torch_cuda
    n = 1 << 13
    e = graphgen.rmat_edges(13, 16, seed=4)
    og, g = build_pair(e, n)
    r = int(graphgen.pick_roots(1, n, 1, og.degree())[0])
    p, l = g.bfs(r)  # numpy outputs: the library copies back and synchronises
    assert_same((l, p), og.bfs(r), "host buffers")
    pp = torch.empty(n, dtype=torch.int32).pin_memory()
    ll = torch.empty(n, dtype=torch.int32).pin_memory()
    g.bfs(r, pp, ll)
    assert_same((ll.numpy(), pp.numpy()), og.bfs(r), "pinned buffers")


def test_uniform_graph(torch_cuda):
    torch = torch_cuda
    n, m = 50000, 50000 * 8
    e = graphgen.uniform_edges(n, m, seed=8)
    og, g = build_pair(e, n)
    roots = graphgen.pick_roots(3, n, 6, og.degree())
    for r, w in zip(roots.tolist(), oracle_many(og, roots)):
        assert_same(bfs_dev(torch, g, r), w, f"uniform root {r}")


def test_edge_cases(torch_cuda):
    torch = torch_cuda
    g = gt.gt_graph_build(np.zeros((0, 2), dtype=np.int64), 5)
    st = g.stats()
    assert st["nnz"] == 0 and st["n_class"][VERTEX_ZERO] == 5
    l, p = bfs_dev(torch, g, 3)
    assert l.tolist() == [-1, -1, -1, 0, -1] and p.tolist() == [-1, -1, -1, 3, -1]
    g1 = gt.gt_graph_build(np.array([[0, 0]], dtype=np.int64), 1)
    l, p = bfs_dev(torch, g1, 0)
    assert l.tolist() == [0] and p.tolist() == [0]
    with pytest.raises(gt.GtError) as ei:
        gt.gt_graph_build(np.array([[0, 5]], dtype=np.int64), 5)
    assert ei.value.code == gt.GT_EINVAL
    with pytest.raises(gt.GtError):
        g.bfs(5)
    with pytest.raises(gt.GtError):
        g.bfs(-1)
    gk = gt.gt_graph_build(np.array([[0, 1]], dtype=np.int64), 2, keep_plain=False)
    with pytest.raises(gt.GtError) as ei:
        gk.bfs_plain(0)
    assert ei.value.code == gt.GT_ENOTSUP
    # a graph larger than one bitmap chunk with a ragged tail and few edges
    n = 4096 * 3 + 77
    e = np.array([(i, i + 1) for i in range(0, n - 1, 2)] + [(n - 2, n - 1), (0, n - 1)], dtype=np.int64)
    og, g = build_pair(e, n)
    for r in (0, n - 1, n - 2, 4096):
        for plain in (False, True):
            g.set_tuning(force_direction=2)
            assert_same(bfs_dev(torch, g, r, plain), og.bfs(r), f"ragged root {r}")


def test_scale22_config(torch_cuda):
    """Core/edge-tree BFS, R-MAT scale 22, 64 seeded roots, one at a time: oracle parity + certificate."""
    torch = torch_cuda
    scale, n = 22, 1 << 22
    e = graphgen.rmat_edges(scale, 16, seed=1)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(2, n, 64, og.degree())
    want = oracle_many(og, roots)
    ed = torch.from_numpy(e).cuda()
    for i, (r, w) in enumerate(zip(roots.tolist(), want)):
        got = bfs_dev(torch, g, r)
        assert_same(got, w, f"s22 root {r}")
        if i < 4:
            assert_same(bfs_dev(torch, g, r, plain=True), w, f"s22 plain root {r}")
            lv = torch.from_numpy(got[0]).cuda()
            pa = torch.from_numpy(got[1]).cuda()
            bfs_certificate(ed, lv, pa, r)
            assert gt.gt_count_traversed(ed, lv) == int(((got[0][e[:, 0]] >= 0) & (got[0][e[:, 1]] >= 0)).sum())


def test_bfs_roots_pipelined_outputs(torch_cuda):
    torch = torch_cuda
    # gt_bfs_roots: several roots in one call with pinned host, pageable host and device
    # outputs mixed (the two device staging pairs are reused more than once); every result
    # equals the oracle's
    s = 13
    n = 1 << s
    e = graphgen.rmat_edges(s, 16, seed=61)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(62, n, 7, og.degree()).tolist()
    kinds = ["pinned", "pageable", "device", "pinned", "pinned", "pageable", "device"]
    bufs = []
    for k in kinds:
        if k == "pinned":
            bufs.append((torch.full((n,), 7, dtype=torch.int32).pin_memory(), torch.full((n,), 7, dtype=torch.int32).pin_memory()))
        elif k == "pageable":
            bufs.append((np.full(n, 7, dtype=np.int32), np.full(n, 7, dtype=np.int32)))
        else:
            bufs.append((torch.full((n,), 7, dtype=torch.int32, device="cuda"),
                         torch.full((n,), 7, dtype=torch.int32, device="cuda")))
    g.bfs_roots(roots, [b[0] for b in bufs], [b[1] for b in bufs])
    torch.cuda.synchronize()
    for r, k, (p, l) in zip(roots, kinds, bufs):
        want_l, want_p = og.bfs(r)
        got_p = p if isinstance(p, np.ndarray) else p.cpu().numpy()
        got_l = l if isinstance(l, np.ndarray) else l.cpu().numpy()
        assert np.array_equal(got_l, want_l), f"level mismatch (root {r}, {k})"
        assert np.array_equal(got_p, want_p), f"parent mismatch (root {r}, {k})"
    with pytest.raises(gt.GtError):
        g.bfs_roots([n], [bufs[0][0]], [bufs[0][1]])  # root out of range
    with pytest.raises(gt.GtError):
        g.bfs_roots([0], [bufs[0][0]], [bufs[2][1]])  # host parent, device level
    g.free()

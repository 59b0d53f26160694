"""Checkpoint of a built graph (gt_graph_save / gt_graph_load): a loaded graph has the
saved graph's statistics, classes and degrees, and its traversals (edge-tree, plain and
batched) equal the oracle's; a damaged file is refused without keeping anything."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from helpers import oracle_many
from oracle import OracleGraph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mh", [0, 1])
def test_save_load_round_trip(tmp_path, mh):
    import torch
    n = 1 << 13
    e = graphgen.rmat_edges(13, 16, seed=51)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n, mh=mh)
    g.set_tuning(bu_thread_scan=16)
    path = str(tmp_path / "g.gtg")
    gt.gt_graph_save(g, path)
    h = gt.gt_graph_load(path)
    a, b = g.stats(), h.stats()
    for k in ("n", "m", "nnz", "n_core", "nnz_core", "n_class", "mh", "height"):
        assert a[k] == b[k], k
    assert np.array_equal(g.vertex_type(), h.vertex_type())
    assert np.array_equal(g.degree(), h.degree())
    assert h.get_tuning().bu_thread_scan == 16
    g.free()
    roots = graphgen.pick_roots(52, n, 12, og.degree()).tolist()
    want = oracle_many(og, roots)
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    for r, (wl, wp) in zip(roots, want):
        for plain in (False, True):
            h.bfs(r, p, lv, plain=plain)
            torch.cuda.synchronize()
            assert np.array_equal(lv.cpu().numpy(), wl) and np.array_equal(p.cpu().numpy(), wp), (r, plain)
    P = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
    L = torch.empty_like(P)
    gt.gt_bfs_batch([h], [roots], [P], [L])
    torch.cuda.synchronize()
    for i, (wl, wp) in enumerate(want):
        assert np.array_equal(L[i].cpu().numpy(), wl) and np.array_equal(P[i].cpu().numpy(), wp)


def test_save_load_large_core_batch(tmp_path):
    """R-MAT scale 21 (core above 2^19 vertices, so its batched work lists include the
    medium-row list): the loaded graph's batched traversal equals the saved graph's, bit
    for bit."""
    import torch
    n = 1 << 21
    e = graphgen.rmat_edges(21, 16, seed=54)
    g = gt.gt_graph_build(e, n)
    assert g.stats()["n_core"] >= 1 << 19
    path = str(tmp_path / "g21.gtg")
    gt.gt_graph_save(g, path)
    h = gt.gt_graph_load(path)
    roots = graphgen.pick_roots(55, n, 64, g.degree()).tolist()
    outs = []
    for x in (g, h):
        P = torch.empty((len(roots), n), dtype=torch.int32, device="cuda")
        L = torch.empty_like(P)
        gt.gt_bfs_batch([x], [roots], [P], [L])
        torch.cuda.synchronize()
        outs.append((P, L))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    g.free()
    h.free()


def test_load_refuses_damaged_files(tmp_path):
    import torch
    n = 1 << 10
    e = graphgen.rmat_edges(10, 16, seed=53)
    g = gt.gt_graph_build(e, n)
    path = tmp_path / "g.gtg"
    gt.gt_graph_save(g, str(path))
    data = path.read_bytes()
    torch.cuda.synchronize()
    gt.gt_graph_load(str(path)).free()  # warm-up of the load path
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    bad = [data[: len(data) // 2], b"not a graph" + data[11:], data[:8] + b"\x09" + data[9:]]
    for i, blob in enumerate(bad):
        q = tmp_path / f"bad{i}.gtg"
        q.write_bytes(blob)
        with pytest.raises(gt.GtError) as ei:
            gt.gt_graph_load(str(q))
        assert ei.value.code == gt.GT_EIO
    with pytest.raises(gt.GtError) as ei:
        gt.gt_graph_load(str(tmp_path / "missing.gtg"))
    assert ei.value.code == gt.GT_EIO
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0

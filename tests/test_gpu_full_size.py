"""Full-size configurations, in the launch configuration the benchmark times (CUDA-graph level
loop, default tuning, device-resident tuples and outputs): R-MAT scale 26 single-root
edge-tree BFS and R-MAT scale 24 batches of 64 roots. Each answer is checked by the
size-independent BFS certificate (levels are hop distances, every parent is the smallest
neighbour one level up) and by agreement between independent paths (edge-tree vs plain BFS;
batched lanes vs single-root calls)."""
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from helpers import bfs_certificate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def device_rmat(torch, scale):
    n, m = 1 << scale, 16 << scale
    e = torch.empty((m, 2), dtype=torch.int64, device="cuda")
    graphgen.rmat_edges_device(e.data_ptr(), scale, m, seed=1)
    torch.cuda.synchronize()
    return e, n


def test_scale26_certificate_and_plain_agreement(torch):
    e, n = device_rmat(torch, 26)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(2, n, 64, g.degree()).tolist()
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    l = torch.empty(n, dtype=torch.int32, device="cuda")
    p2 = torch.empty_like(p)
    l2 = torch.empty_like(l)
    # the first roots of the benchmark's sequence plus two whose level 2 is a hub frontier
    for r in (roots[0], roots[1], roots[19], roots[45]):
        g.bfs(r, p, l)
        g.bfs_plain(r, p2, l2)
        torch.cuda.synchronize()
        reached = bfs_certificate(e, l, p, r)
        assert reached > n // 3, f"root {r}: only {reached} vertices reached"
        assert torch.equal(l, l2) and torch.equal(p, p2), f"root {r}: edge-tree and plain BFS differ"
    g.free()


def test_scale24_batch_lanes(torch):
    e, n = device_rmat(torch, 24)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(2, n, 64, g.degree()).tolist()
    P = torch.empty((64, n), dtype=torch.int32, device="cuda")
    L = torch.empty((64, n), dtype=torch.int32, device="cuda")
    gt.gt_bfs_batch([g], [roots], [P], [L])
    torch.cuda.synchronize()
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    l = torch.empty(n, dtype=torch.int32, device="cuda")
    for lane in (0, 17, 40, 63):
        g.bfs(roots[lane], p, l)
        torch.cuda.synchronize()
        assert torch.equal(L[lane], l) and torch.equal(P[lane], p), f"lane {lane} differs from gt_bfs"
    bfs_certificate(e, L[5], P[5], roots[5])
    g.free()

"""Failure detection without a GPU fault: the bounded grid-barrier waits of the batched
persistent launch, and device allocations that fail during graph construction. A barrier that waits for arrivals that never come (set through the
test hook gt_test_batch_barrier) must give up after its poll bound, every CTA must leave
the kernel, the call must report GT_ETIMEOUT, and the device must stay usable: the next
launch with the default bound is bit-identical to the oracle, and so is a single-root
traversal in between."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from oracle import OracleGraph

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_the_device_stays_usable():
    import torch
    n = 1 << 12
    e = graphgen.rmat_edges(12, 16, seed=31)
    og = OracleGraph(e, n)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(5, n, 8, og.degree()).tolist()
    P = torch.empty((8, n), dtype=torch.int32, device="cuda")
    L = torch.empty((8, n), dtype=torch.int32, device="cuda")
    try:
        gt.gt_test_batch_barrier(polls=2000, extra=1)  # one arrival that never comes
        for _ in range(2):  # the captured launch is replayed with the same bound
            with pytest.raises(gt.GtError) as ei:
                gt.gt_bfs_batch([g], [roots], [P], [L])
            assert ei.value.code == gt.GT_ETIMEOUT and "barrier" in str(ei.value)
    finally:
        gt.gt_test_batch_barrier(0, 0)
    torch.cuda.synchronize()  # no kernel is left waiting
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    g.bfs(roots[0], p, lv)
    wl, wp = og.bfs(roots[0])
    assert np.array_equal(lv.cpu().numpy(), wl) and np.array_equal(p.cpu().numpy(), wp)
    P.fill_(-7)
    L.fill_(-7)
    gt.gt_bfs_batch([g], [roots], [P], [L])
    torch.cuda.synchronize()
    for i, r in enumerate(roots):
        wl, wp = og.bfs(r)
        assert np.array_equal(L[i].cpu().numpy(), wl), f"level of root {r} after the timed-out launch"
        assert np.array_equal(P[i].cpu().numpy(), wp), f"parent of root {r} after the timed-out launch"


def test_allocation_failure_during_build_frees_everything():
    """An allocation that fails at several points of graph construction (injected on the
    host): gt_graph_build returns GT_ENOMEM, the device memory it took is given back, and
    the next build is complete and correct."""
    import torch
    n = 1 << 12
    e = graphgen.rmat_edges(12, 16, seed=33)
    og = OracleGraph(e, n)
    gt.gt_graph_build(e, n).free()  # warm-up: contexts and kernels in place
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    try:
        for after in (0, 1, 4, 11, 25):
            gt.gt_test_fail_alloc(after)
            with pytest.raises(gt.GtError) as ei:
                gt.gt_graph_build(e, n)
            assert ei.value.code == gt.GT_ENOMEM and "injected" in str(ei.value)
    finally:
        gt.gt_test_fail_alloc(-1)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"{free0 - free1} bytes of device memory not given back"
    g = gt.gt_graph_build(e, n)
    r = int(graphgen.pick_roots(34, n, 1, og.degree())[0])
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    g.bfs(r, p, lv)
    wl, wp = og.bfs(r)
    assert np.array_equal(lv.cpu().numpy(), wl) and np.array_equal(p.cpu().numpy(), wp)

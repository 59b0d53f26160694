"""The traversal that allocates nothing (gt_bfs_csr_noalloc), for callers that may not
allocate device memory when they run a query (a memory plan fixed at start-up, or a
plug-in that only gets its inputs and outputs). Its results must equal those of the
allocating entry point gt_bfs_plain and of the CPU oracle, bit for bit, on calls in a row
(the fixed scratch keeps the previous call's contents, so later calls check that it is
cleared): the hand-made graphs with every root, a graph whose vertex count is not a
multiple of the 4096-vertex bitmap chunk, and an R-MAT graph of exactly 262,144 vertices,
the largest the scratch holds, followed by smaller graphs.
This file sorts last so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from oracle import OracleGraph
from test_gpu_parity import HAND

pytestmark = pytest.mark.gpu


def dev_csr(torch, og):
    """The oracle's CSR of the input tuples as device tensors (input only; col padded by one
    entry so that an edgeless graph still passes a non-null column pointer)."""
    row_h, col_h = og.csr()
    row = torch.from_numpy(row_h).cuda()
    col = torch.from_numpy(np.concatenate([col_h, np.zeros(1, np.int32)])).cuda()
    return row, col


def noalloc(torch, row, col, n, r):
    p = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    l = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    gt.gt_bfs_csr_noalloc(row, col, n, r, p, l)
    torch.cuda.synchronize()
    return l, p


def assert_oracle(l, p, want, what):
    wl, wp = want
    gl, gp = l.cpu().numpy(), p.cpu().numpy()
    assert np.array_equal(gl, wl), f"{what}: level differs at {np.flatnonzero(gl != wl)[:8].tolist()}"
    assert np.array_equal(gp, wp), f"{what}: parent differs at {np.flatnonzero(gp != wp)[:8].tolist()}"


def test_noalloc_equals_allocating_entry_point_twice():
    import torch
    assert torch.cuda.is_available()
    scale = 16
    n = 1 << scale
    e = graphgen.rmat_edges(scale, 16, seed=12)
    row_h, col_h = OracleGraph(e, n).csr()  # input CSR only; expected values come from gt_bfs_plain
    row = torch.from_numpy(row_h).cuda()
    col = torch.from_numpy(np.ascontiguousarray(col_h)).cuda()
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(13, n, 2, np.diff(row_h)).tolist()
    for r in roots:  # two calls in a row
        p = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        l = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        gt.gt_bfs_csr_noalloc(row, col, n, r, p, l)
        wp = torch.empty(n, dtype=torch.int32, device="cuda")
        wl = torch.empty(n, dtype=torch.int32, device="cuda")
        g.bfs_plain(r, wp, wl)
        torch.cuda.synchronize()
        assert torch.equal(l, wl), f"level differs for root {r}"
        assert torch.equal(p, wp), f"parent differs for root {r}"


def test_noalloc_matches_oracle_across_sizes():
    """Largest graph first (262,144 vertices), then a ragged one, then the hand-made graphs
    with every root: each call starts from what the previous, larger call left behind."""
    import torch
    cases = []
    e18 = graphgen.rmat_edges(18, 16, seed=5)
    og18 = OracleGraph(e18, 1 << 18)
    cases.append(("rmat s18", og18, 1 << 18, graphgen.pick_roots(6, 1 << 18, 3, og18.degree()).tolist()))
    n = 4096 * 3 + 77
    eu = graphgen.uniform_edges(n, 4 * n, seed=7)
    ogu = OracleGraph(eu, n)
    isolated = int(np.flatnonzero(ogu.degree() == 0)[0]) if (ogu.degree() == 0).any() else 0
    cases.append(("uniform ragged", ogu, n, [0, n - 1, 4096, isolated]))
    for name in sorted(HAND):
        pairs, nh = HAND[name]
        ogh = OracleGraph(np.array(pairs, dtype=np.int64).reshape(-1, 2), nh)
        cases.append((name, ogh, nh, list(range(nh))))
    for name, og, nv, roots in cases:
        row, col = dev_csr(torch, og)
        for r in roots:
            l, p = noalloc(torch, row, col, nv, r)
            assert_oracle(l, p, og.bfs(r), f"{name} root {r}")


def test_noalloc_allocates_no_device_memory():
    """Free device memory is the same before and after calls on two graphs of different
    sizes (the scratch array and the kernels are in place after the first call)."""
    import torch
    e = graphgen.rmat_edges(14, 16, seed=9)
    og = OracleGraph(e, 1 << 14)
    row, col = dev_csr(torch, og)
    eh = np.array(HAND["lollipop"][0], dtype=np.int64)
    ogh = OracleGraph(eh, HAND["lollipop"][1])
    rowh, colh = dev_csr(torch, ogh)
    roots = graphgen.pick_roots(3, 1 << 14, 2, og.degree()).tolist()
    outs = [torch.empty(1 << 14, dtype=torch.int32, device="cuda") for _ in range(2)]
    gt.gt_bfs_csr_noalloc(row, col, 1 << 14, roots[0], outs[0], outs[1])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for r in roots:
        gt.gt_bfs_csr_noalloc(row, col, 1 << 14, r, outs[0], outs[1])
        gt.gt_bfs_csr_noalloc(rowh, colh, HAND["lollipop"][1], 0, outs[0], outs[1])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = (1 << 18) + 1
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GtError) as ei:
        gt.gt_bfs_csr_noalloc(row, col, n, 0, out, out)
    assert ei.value.code == gt.GT_EINVAL and "capacity" in str(ei.value)


def test_noalloc_rejects_bad_inputs():
    """Buffers of the wrong type or length are refused before the library is called, and
    host memory is refused by the library itself."""
    import torch
    n = 8
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    row[n] = 4
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        gt.gt_bfs_csr_noalloc(row.int(), col, n, 0, out, out)        # int32 row offsets
    with pytest.raises(ValueError):
        gt.gt_bfs_csr_noalloc(row[:n], col, n, 0, out, out)          # one offset short
    with pytest.raises(ValueError):
        gt.gt_bfs_csr_noalloc(row, col[:3], n, 0, out, out)          # col shorter than row[n]
    with pytest.raises(gt.GtError) as ei:
        gt.gt_bfs_csr_noalloc(row.cpu(), col.cpu(), n, 0, out, out)  # host memory
    assert ei.value.code == gt.GT_EINVAL

"""The traversal that allocates nothing (gt_bfs_csr_noalloc), for callers that may not
allocate device memory when they run a query (a memory plan fixed at start-up, or a
plug-in that only gets its inputs and outputs). Its results must equal those of the
allocating entry point gt_bfs_plain, bit for bit, on two calls in a row (the fixed scratch
keeps the previous call's contents, so the second call checks that it is cleared).
This file sorts last so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt
from oracle import OracleGraph

pytestmark = pytest.mark.gpu


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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    n = (1 << 18) + 1
    row = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GtError) as ei:
        gt.gt_bfs_csr_noalloc(row, col, n, 0, out, out)
    assert ei.value.code == gt.GT_EINVAL and "capacity" in str(ei.value)

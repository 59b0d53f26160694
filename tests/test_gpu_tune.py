"""The autotuner picks a setting and keeps it in the handle; results never change."""
import numpy as np
import pytest

import graphgen
import paper_2009_07463_gb300 as gt

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results():
    n = 1 << 15
    e = graphgen.rmat_edges(15, 16, seed=21)
    g = gt.gt_graph_build(e, n)
    roots = graphgen.pick_roots(22, n, 6, g.degree()).tolist()
    before = [g.bfs(r) for r in roots]
    t = g.autotune(nsample=4, seed=3)
    now = g.get_tuning()
    for f, _ in gt.gt_tuning._fields_:
        assert getattr(t, f) == getattr(now, f)
    assert t.launch_mode == 0 and t.count_work == 0 and t.time_kernels == 0
    assert t.td_warp_min <= t.td_cta_min <= t.td_grid_min
    for r, (p0, l0) in zip(roots, before):
        p1, l1 = g.bfs(r)
        assert np.array_equal(p0, p1) and np.array_equal(l0, l1)

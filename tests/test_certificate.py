"""The size-independent BFS certificate used at full sizes accepts the oracle's answers and
rejects planted mistakes (run on CPU tensors; no GPU needed)."""
import numpy as np
import pytest

import graphgen
from helpers import bfs_certificate
from oracle import OracleGraph

torch = pytest.importorskip("torch")


def test_certificate_accepts_oracle_and_rejects_mistakes():
    n = 1 << 12
    e = graphgen.rmat_edges(12, 16, seed=3)
    og = OracleGraph(e, n)
    root = int(graphgen.pick_roots(1, n, 1, og.degree())[0])
    lv, pa = og.bfs(root)
    et = torch.from_numpy(e)
    bfs_certificate(et, torch.from_numpy(lv), torch.from_numpy(pa), root)
    reached = np.flatnonzero((lv > 1))
    v = int(reached[0])
    # a non-minimal but valid-looking parent
    row, col = og.csr()
    nb = col[row[v]:row[v + 1]]
    ups = nb[lv[nb] == lv[v] - 1]
    bad = pa.copy()
    if ups.size > 1:
        bad[v] = ups.max()
        with pytest.raises(AssertionError):
            bfs_certificate(et, torch.from_numpy(lv), torch.from_numpy(bad), root)
    # a level off by one
    badl = lv.copy()
    badl[v] += 1
    with pytest.raises(AssertionError):
        bfs_certificate(et, torch.from_numpy(badl), torch.from_numpy(pa), root)
    # an unreached vertex reported reached
    badl = lv.copy()
    un = np.flatnonzero(lv < 0)
    badl[un[0]] = 3
    with pytest.raises(AssertionError):
        bfs_certificate(et, torch.from_numpy(badl), torch.from_numpy(pa), root)

"""Host-side checks of the seeded input generator (no GPU)."""
import numpy as np
import pytest

import graphgen


@pytest.mark.parametrize("scale", list(range(1, 17)))
def test_perm_is_bijection(scale):
    p = graphgen.perm_values(3, scale)
    assert np.array_equal(np.sort(p), np.arange(1 << scale))


def test_quadrant_frequencies_scale1():
    # at scale 1 without scrambling each tuple is one quadrant draw: (0,0) A, (0,1) B, (1,0) C, (1,1) D
    m = 400_000
    e = graphgen.rmat_edges(1, m=m, seed=9, permute=False)
    code = e[:, 0] * 2 + e[:, 1]
    counts = np.bincount(code, minlength=4)
    for c, p in zip(counts, (0.57, 0.19, 0.19, 0.05)):
        sigma = np.sqrt(m * p * (1 - p))
        assert abs(c - m * p) < 6 * sigma


def test_rmat_shape_range_determinism():
    e1 = graphgen.rmat_edges(10, 16, seed=4)
    e2 = graphgen.rmat_edges(10, 16, seed=4)
    e3 = graphgen.rmat_edges(10, 16, seed=5)
    assert e1.shape == (16 << 10, 2) and e1.dtype == np.int64
    assert e1.min() >= 0 and e1.max() < 1 << 10
    assert np.array_equal(e1, e2) and not np.array_equal(e1, e3)


def test_rmat_unscrambled_skew():
    # without scrambling, vertex 0 (all-A path) is the expected hub
    e = graphgen.rmat_edges(12, 16, seed=2, permute=False)
    deg = np.bincount(e.ravel(), minlength=1 << 12)
    assert deg.argmax() == 0
    # scrambling permutes ids without changing the degree multiset
    es = graphgen.rmat_edges(12, 16, seed=2, permute=True)
    assert np.array_equal(np.sort(np.bincount(es.ravel(), minlength=1 << 12)), np.sort(deg))


def test_uniform_edges():
    n, m = 1000, 200_000
    e = graphgen.uniform_edges(n, m, seed=1)
    assert e.min() >= 0 and e.max() < n
    cnt = np.bincount(e.ravel(), minlength=n)
    assert abs(cnt.mean() - 2 * m / n) < 1e-9
    assert cnt.std() < 4 * np.sqrt(2 * m / n)


def test_pick_roots():
    deg = np.zeros(5000, dtype=np.int64)
    deg[::3] = 2
    r1 = graphgen.pick_roots(8, 5000, 64, deg)
    r2 = graphgen.pick_roots(8, 5000, 64, deg)
    assert np.array_equal(r1, r2)
    assert len(set(r1.tolist())) == 64 and (deg[r1] >= 1).all()
    with pytest.raises(ValueError):
        graphgen.pick_roots(8, 10, 3, np.array([1, 0, 0, 0, 0, 0, 0, 0, 0, 1]))

"""The seeded generators produce simple graphs in the library's CSR contract,
deterministically."""
import numpy as np
import pytest

import graphgen as gg


def assert_simple_csr(rp, ci):
    n = len(rp) - 1
    assert rp[0] == 0 and rp[-1] == len(ci)
    assert (np.diff(rp) >= 0).all()
    if len(ci) == 0:
        return
    assert ci.min() >= 0 and ci.max() < n
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert not (rows == ci).any(), "self-loop"
    key = rows.astype(np.int64) * n + ci
    assert (np.diff(key) > 0).all(), "rows not strictly increasing"
    rev = np.sort(ci.astype(np.int64) * n + rows)
    assert np.array_equal(rev, key), "not symmetric"


@pytest.mark.parametrize("make", [
    lambda s: gg.er(500, 0.02, s),
    lambda s: gg.er_mean_degree(20000, 8, s),
    lambda s: gg.rmat(11, 16, seed=s),
    lambda s: gg.chunglu(3000, 2.5, 8.0, s),
])
def test_simple_and_deterministic(make):
    a = make(3)
    b = make(3)
    c = make(4)
    assert_simple_csr(*a)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))


def test_er_edge_count():
    n, p = 2000, 0.01
    rp, ci = gg.er(n, p, 1)
    mean = p * n * (n - 1) / 2
    assert abs(len(ci) // 2 - mean) < 5 * np.sqrt(mean)


def test_rmat_skew():
    rp, ci = gg.rmat(14, 16, seed=2)
    d = np.diff(rp)
    assert d.max() > 50 * d.mean()          # hubs
    assert (d == 0).sum() > 0               # isolated vertices exist


def test_chunglu_mean_degree():
    rp, ci = gg.chunglu(5000, 2.5, 8.0, 1)
    assert 5.0 < len(ci) / 5000 < 9.0


def test_from_edges_drops_loops_and_duplicates():
    rp, ci = gg.from_edges(4, [(0, 1), (1, 0), (2, 2), (1, 3), (1, 3)])
    assert rp.tolist() == [0, 1, 3, 3, 4]
    assert ci.tolist() == [1, 0, 3, 1]


def test_batch_sizes_range():
    s = gg.batch_sizes(4000, 50, 5000, seed=1)
    assert s.min() >= 50 and s.max() <= 5000
    assert 700 < s.mean() < 1400

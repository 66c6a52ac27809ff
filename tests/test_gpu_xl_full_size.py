"""Full-size parity (the two large single-graph configurations): every row
against invariants that hold at any size, and sampled rows against the
oracle's per-vertex mode. Kept in a file of its own so that it runs after the
smaller GPU tests.

The oracle's per-vertex Stage III costs O(d^2) pair tests plus, for every
path x-y-z, an intersection of the rows of y and z; a sampled vertex whose
neighbours are hubs of degree ~1e5 would take hours. The sample is therefore
random vertices of degree at most 64, the 20 largest vertices of degree at
most 300, and 20 low-degree neighbours of the largest hub.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import cheap_sum_checks
from test_gpu_parity import assert_same, gpu_count

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_29651_gb300 as ni
    ni.build()
    return ni


def _sample(rp, ci, nsample, seed):
    d = np.diff(rp)
    rng = np.random.default_rng(seed)
    low = np.flatnonzero((d >= 1) & (d <= 64))
    pick = set(rng.choice(low, size=min(nsample, len(low)), replace=False).tolist())
    order = np.argsort(-d, kind="stable")
    pick.update(int(v) for v in order[d[order] <= 300][:20])
    top = int(order[0])
    nb = ci[rp[top]:rp[top + 1]]
    nb = nb[d[nb] <= 64]
    pick.update(int(v) for v in rng.choice(nb, size=min(20, len(nb)), replace=False))
    return np.array(sorted(pick), dtype=np.int32)


def _full_size_check(ni, rp, ci, nsample, seed):
    got = gpu_count(ni, rp, ci)
    assert cheap_sum_checks(rp, got) == []
    verts = _sample(rp, ci, nsample, seed)
    assert_same(got[verts], oracle.count_vertices(rp, ci, verts), "sampled rows")
    return got


def test_er_1e6_sampled(ni):
    rp, ci = gg.er_mean_degree(1_000_000, 32, 1)
    _full_size_check(ni, rp, ci, 300, 11)


def test_rmat22_sampled(ni):
    rp, ci = gg.rmat(22, 16, seed=1)
    _full_size_check(ni, rp, ci, 150, 12)

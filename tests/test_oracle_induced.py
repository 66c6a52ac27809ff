"""Pins for induced orbit counts (the variant of Sec. 5 that ORCA computes):
closed forms, the paper's three printed induced equations, and the relation
non-induced = overlap matrix x induced, the matrix found by brute force."""
import itertools
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import random_small_graphs


def _csr(n, edges):
    if edges:
        return gg.from_edges(n, edges)
    return np.zeros(n + 1, np.int32), np.zeros(0, np.int32)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7])
def test_induced_complete_graph(n):
    m = n - 1
    row = [0] * 15
    row[0], row[3], row[14] = m, comb(m, 2), comb(m, 3)
    assert np.array_equal(oracle.induced_count(*gg.complete(n)), np.tile(row, (n, 1)))
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    assert np.array_equal(np.array(oracle.brute_count(n, edges, induced=True)), np.tile(row, (n, 1)))


def test_induced_c4_and_chordless_graphs():
    c4 = oracle.induced_count(*gg.cycle(4))
    assert np.array_equal(c4, np.tile([2, 2, 1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0], (4, 1)))
    # no chords: induced equals non-induced
    for g in (gg.cycle(9), gg.path(7), gg.star(6)):
        assert np.array_equal(oracle.induced_count(*g), oracle.count(*g))


def test_printed_induced_equations():
    """The induced equations printed in Sec. 5: psi'13 = f13/2 - 3 psi14;
    psi'11 = (f11 - f13)/2 + 3 psi14; psi'10 = f10 - f13 + 6 psi14, with
    the non-induced f* read back from
    Eqs. o13, o12, o11, o10: f13 = 2 psi13, f12 = psi12, f11 = 2 psi11 - f13,
    f10 = psi10 - 2 psi12."""
    for rp, ci in (gg.er(300, 0.1, 2), gg.rmat(9, 16, seed=4), gg.er(60, 0.5, 5)):
        nind = oracle.count(rp, ci)
        ind = oracle.induced_count(rp, ci)
        f13 = 2 * nind[:, 13]
        f11 = 2 * nind[:, 11] - f13
        f10 = nind[:, 10] - 2 * nind[:, 12]
        assert np.array_equal(ind[:, 13], f13 // 2 - 3 * nind[:, 14])
        assert np.array_equal(ind[:, 11], (f11 - f13) // 2 + 3 * nind[:, 14])
        assert np.array_equal(ind[:, 10], f10 - f13 + 6 * nind[:, 14])


def _overlap_matrix():
    """O[k][j]: spanning non-induced graphlets with x in orbit k inside the
    induced graphlet with x in orbit j, by brute force on representatives."""
    reps = {  # (n, edges, vertex) realising each orbit as an induced graphlet
        0: (2, [(0, 1)], 0), 1: (3, [(0, 1), (1, 2)], 0), 2: (3, [(0, 1), (1, 2)], 1),
        3: (3, [(0, 1), (1, 2), (0, 2)], 0),
        4: (4, [(0, 1), (1, 2), (2, 3)], 0), 5: (4, [(0, 1), (1, 2), (2, 3)], 1),
        6: (4, [(0, 1), (0, 2), (0, 3)], 1), 7: (4, [(0, 1), (0, 2), (0, 3)], 0),
        8: (4, [(0, 1), (1, 2), (2, 3), (3, 0)], 0),
        9: (4, [(0, 1), (1, 2), (0, 2), (2, 3)], 3), 10: (4, [(0, 1), (1, 2), (0, 2), (2, 3)], 0),
        11: (4, [(0, 1), (1, 2), (0, 2), (2, 3)], 2),
        12: (4, [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], 0),
        13: (4, [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)], 2),
        14: (4, [(a, b) for a, b in itertools.combinations(range(4), 2)], 0),
    }
    O = np.zeros((15, 15), dtype=np.int64)
    for j, (n, edges, x) in reps.items():
        ind = np.array(oracle.brute_count(n, edges, induced=True))
        assert ind[x, j] == 1 and ind[x].sum() - ind[x, :3].sum() * (n == 4) >= 1
        full = np.array(oracle.brute_count(n, edges))
        # only the subgraphs on all n vertices: orbits of the n-vertex graphlets
        lo, hi = {2: (0, 1), 3: (1, 4), 4: (4, 15)}[n]
        O[lo:hi, j] = full[x, lo:hi]
    return O


def test_noninduced_is_overlap_times_induced():
    O = _overlap_matrix()
    assert np.array_equal(np.diag(O), np.ones(15))
    assert np.array_equal(O, np.triu(O))
    for n, edges in random_small_graphs(80, 9, seed=31):
        rp, ci = _csr(n, edges)
        assert np.array_equal(oracle.count(rp, ci), oracle.induced_count(rp, ci) @ O.T), (n, edges)

"""Pins for the oracle: brute force, closed forms, hand-worked tables and
orbit-sum invariants. None of these expected values comes from the oracle
itself or from the CUDA path."""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import (cheap_sum_checks, closed_complete, closed_complete_bipartite, closed_cycle,
                     closed_path, closed_star, graphlet_totals, orbit_sums_expected,
                     random_small_graphs, read_golden)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.txt")


def _csr(n, edges):
    if edges:
        return gg.from_edges(n, edges)
    return np.zeros(n + 1, np.int32), np.zeros(0, np.int32)


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("n", range(1, 8))
def test_brute_complete_closed_form(n):
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    psi = np.array(oracle.brute_count(n, edges))
    exp = np.tile(np.maximum(np.array(closed_complete(n)), 0), (n, 1))
    assert np.array_equal(psi, exp)


@pytest.mark.parametrize("k", range(1, 7))
def test_brute_star_closed_form(k):
    psi = np.array(oracle.brute_count(k + 1, [(0, i) for i in range(1, k + 1)]))
    assert np.array_equal(psi, closed_star(k))


@pytest.mark.parametrize("n", range(3, 9))
def test_brute_cycle_closed_form(n):
    psi = np.array(oracle.brute_count(n, [(i, (i + 1) % n) for i in range(n)]))
    assert np.array_equal(psi, closed_cycle(n))


@pytest.mark.parametrize("n", range(1, 9))
def test_brute_path_closed_form(n):
    psi = np.array(oracle.brute_count(n, [(i, i + 1) for i in range(n - 1)]))
    assert np.array_equal(psi, closed_path(n))


@pytest.mark.parametrize("a,b", [(1, 1), (1, 4), (2, 3), (3, 3), (2, 5)])
def test_brute_bipartite_closed_form(a, b):
    psi = np.array(oracle.brute_count(a + b, [(i, a + j) for i in range(a) for j in range(b)]))
    assert np.array_equal(psi, closed_complete_bipartite(a, b))


def test_brute_hand_worked_tables():
    for name, n, edges, table in read_golden(GOLDEN):
        assert np.array_equal(np.array(oracle.brute_count(n, edges)), table), name


# ------------------------------------------- C oracles vs the pins above

def test_golden_tables_all_oracles():
    for name, n, edges, table in read_golden(GOLDEN):
        rp, ci = _csr(n, edges)
        assert np.array_equal(oracle.count(rp, ci), table), name
        assert np.array_equal(oracle.definition_count(rp, ci), table), name


@pytest.mark.parametrize("fn", ["count", "definition_count"])
def test_closed_forms_larger(fn):
    f = getattr(oracle, fn)
    for n in (8, 11):
        rp, ci = gg.complete(n)
        assert np.array_equal(f(rp, ci), np.tile(np.array(closed_complete(n)), (n, 1)))
    for k in (9, 40):
        assert np.array_equal(f(*gg.star(k)), closed_star(k))
    for n in (3, 4, 5, 31):
        assert np.array_equal(f(*gg.cycle(n)), closed_cycle(n))
    for n in (2, 3, 4, 5, 6, 25):
        assert np.array_equal(f(*gg.path(n)), closed_path(n))
    for a, b in ((1, 7), (4, 6), (6, 9)):
        assert np.array_equal(f(*gg.complete_bipartite(a, b)), closed_complete_bipartite(a, b))


def test_random_tiny_graphs_match_brute_force():
    for n, edges in random_small_graphs(250, 9, seed=11):
        rp, ci = _csr(n, edges)
        exp = np.array(oracle.brute_count(n, edges), dtype=np.int64).reshape(n, 15)
        assert np.array_equal(oracle.count(rp, ci), exp), (n, edges)
        assert np.array_equal(oracle.definition_count(rp, ci), exp), (n, edges)
        allv = np.arange(n)
        assert np.array_equal(oracle.count_vertices(rp, ci, allv), exp), (n, edges)
        assert np.array_equal(oracle.definition_count_vertices(rp, ci, allv), exp), (n, edges)


def _medium_graphs():
    yield "er60", gg.er(60, 0.3, 3)
    yield "er200", gg.er(200, 0.08, 4)
    yield "rmat9", gg.rmat(9, 8, seed=5)
    yield "chunglu300", gg.chunglu(300, 2.2, 10.0, 6)
    yield "dense40", gg.er(40, 0.8, 7)


@pytest.mark.parametrize("name,g", list(_medium_graphs()))
def test_paper_form_equals_definition(name, g):
    rp, ci = g
    a = oracle.count(rp, ci)
    d = oracle.definition_count(rp, ci)
    assert np.array_equal(a, d), name
    assert cheap_sum_checks(rp, a) == []
    assert np.array_equal(a.sum(axis=0), orbit_sums_expected(graphlet_totals(rp, ci)))


@pytest.mark.parametrize("name,g", list(_medium_graphs())[:3] + [("rmat11_hubs", gg.rmat(11, 16, seed=13))])
def test_per_vertex_modes_equal_full(name, g):
    rp, ci = g
    n = len(rp) - 1
    a = oracle.count(rp, ci)
    verts = np.arange(0, n, 3)
    assert np.array_equal(oracle.count_vertices(rp, ci, verts), a[verts])
    if name != "rmat11_hubs":   # ESU around a degree-800 hub lists ~1e8 sets
        assert np.array_equal(oracle.definition_count_vertices(rp, ci, verts[:40]), a[verts[:40]])


def test_stage_outputs_against_scipy():
    import scipy.sparse as sp
    rp, ci = gg.rmat(10, 8, seed=9)
    n = len(rp) - 1
    d = np.diff(rp)
    rows = np.repeat(np.arange(n), d)
    A = sp.csr_matrix((np.ones(len(ci), dtype=np.int64), (rows, ci)), shape=(n, n))
    t = np.asarray((A @ A)[rows, ci]).ravel()   # |N(x) ∩ N(y)| at every CSR position
    assert np.array_equal(oracle.stage1_triangles(rp, ci), t.astype(np.int32))
    k4 = oracle.stage2_k4(rp, ci)
    tot = graphlet_totals(rp, ci)
    assert k4.sum() == 4 * tot["k4"]


def test_orbit_sums_er2000():
    rp, ci = gg.er(2000, 0.01, 1)
    a = oracle.count(rp, ci)
    assert np.array_equal(a.sum(axis=0), orbit_sums_expected(graphlet_totals(rp, ci)))
    assert cheap_sum_checks(rp, a) == []


# ------------------------------------------------ the pins catch mistakes

def _pin_suite_detects(run):
    """True if `run(rp, ci)` disagrees with brute force or a closed form."""
    for n, edges in random_small_graphs(60, 8, seed=23):
        rp, ci = _csr(n, edges)
        exp = np.array(oracle.brute_count(n, edges), dtype=np.int64).reshape(n, 15)
        if not np.array_equal(run(rp, ci), exp):
            return True
    for name, n, edges, table in read_golden(GOLDEN):
        if not np.array_equal(run(*_csr(n, edges)), table):
            return True
    return not np.array_equal(run(*gg.complete(6)), np.tile(np.array(closed_complete(6)), (6, 1)))


@pytest.mark.parametrize("mutation", range(1, oracle.N_MUTATIONS + 1))
def test_planted_equation_mistake_is_detected(mutation):
    def run(rp, ci):
        try:
            return oracle.count(rp, ci, mutation=mutation)
        except RuntimeError:
            return None
    assert _pin_suite_detects(run)


@pytest.mark.parametrize("flag", [oracle.READ_F69_EYZ, oracle.READ_NEIGH_NO_RESET,
                                  oracle.READ_FIG3B_ORDERED])
def test_rejected_readings_fail_the_pins(flag):
    def run(rp, ci):
        try:
            return oracle.count(rp, ci, flags=flag)
        except RuntimeError:
            return None
    assert _pin_suite_detects(run)


def test_unmutated_oracle_passes_pin_suite():
    assert not _pin_suite_detects(lambda rp, ci: oracle.count(rp, ci))

"""CUDA path vs the oracle, element by element (integers: bit-exact).

Every call goes through the C ABI (paper_2606_29651_gb300 is a ctypes
binding of libniorca.so)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import (cheap_sum_checks, closed_complete, closed_complete_bipartite, closed_cycle, closed_path,
                     closed_star, random_small_graphs)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_29651_gb300 as ni
    ni.build()
    return ni


def gpu_count(ni, rp, ci):
    dev = torch.device("cuda:0")
    r = torch.from_numpy(np.ascontiguousarray(rp, dtype=np.int32)).to(dev)
    c = torch.from_numpy(np.ascontiguousarray(ci, dtype=np.int32)).to(dev)
    out = ni.count(r, c)
    ni.check()
    return out.cpu().numpy()


def assert_same(got, exp, what):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        v, k = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches; first vertex {v} orbit {k}: "
                             f"got {got[v, k]} expected {exp[v, k]}; row got {got[v].tolist()} exp {exp[v].tolist()}")


def test_tiny_random_graphs_vs_brute_force(ni):
    for n, edges in random_small_graphs(120, 10, seed=101):
        rp, ci = gg.from_edges(n, edges) if edges else (np.zeros(n + 1, np.int32), np.zeros(0, np.int32))
        exp = np.array(oracle.brute_count(n, edges), dtype=np.int64).reshape(n, 15)
        assert_same(gpu_count(ni, rp, ci), exp, f"n={n} edges={edges}")


def test_closed_forms(ni):
    for n in (2, 3, 4, 5, 12, 40, 100, 300):
        assert_same(gpu_count(ni, *gg.complete(n)), np.tile(np.array(closed_complete(n)), (n, 1)), f"K{n}")
    for k in (1, 2, 3, 50, 3000):
        assert_same(gpu_count(ni, *gg.star(k)), closed_star(k), f"star{k}")
    for n in (3, 4, 5, 1000):
        assert_same(gpu_count(ni, *gg.cycle(n)), closed_cycle(n), f"C{n}")
    for n in (2, 5, 777):
        assert_same(gpu_count(ni, *gg.path(n)), closed_path(n), f"P{n}")
    for a, b in ((1, 1), (3, 7), (40, 60), (2, 12000), (3, 9000)):
        assert_same(gpu_count(ni, *gg.complete_bipartite(a, b)), closed_complete_bipartite(a, b), f"K{a},{b}")


def test_complete_graphs_across_triangle_tiers(ni):
    # K1040: out-degrees up to 1039 use the 1152-row bit matrix of the
    # 1024-thread tier; K1200: out-degrees above 1152 take its probing K4 path
    for n in (1040, 1200):
        assert_same(gpu_count(ni, *gg.complete(n)), np.tile(np.array(closed_complete(n)), (n, 1)), f"K{n}")


@pytest.mark.parametrize("pad", [0, (1 << 21) + 5000 - 10000])
def test_four_cycle_warp_tiers_both_table_kinds(ni, pad):
    # An ER core (n = 10^4, mean degree 40) puts 4-cycle roots in both warp
    # tiers and the 4-warp tiers above them. Isolated vertices beyond 2^21
    # leave a packed word 10 count bits, so that every tier counts in split
    # (key, count) tables instead of packed ones.
    import bench

    rp, ci = gg.er_mean_degree(10000, 40, 7)
    exp = np.zeros((10000 + pad, 15), np.int64)
    exp[:10000] = oracle.count(rp, ci)
    rpf = np.concatenate([rp, np.full(pad, rp[-1], rp.dtype)])
    tiers = bench.algorithmic_bytes(rpf, ci)["per_kernel"]
    assert tiers["k_c4_warp"] > 0 and tiers["k_c4_warp_big"] > 0 and tiers["k_c4_mid"] > 0
    assert_same(gpu_count(ni, rpf, ci), exp, f"ER core + {pad} isolated vertices")


@pytest.mark.parametrize("name,make", [
    ("er2000", lambda: gg.er(2000, 0.01, 1)),
    ("rmat12", lambda: gg.rmat(12, 16, seed=3)),
    ("star3000", lambda: gg.star(3000)),          # a row of the long-row class
    ("k300", lambda: gg.complete(300)),
])
def test_host_buffers_equal_device_buffers(ni, name, make):
    # niorca_count_host reads the pinned CSR and writes the pinned counts in place
    rp, ci = make()
    h_rp = torch.from_numpy(np.ascontiguousarray(rp, np.int32)).pin_memory()
    h_ci = torch.from_numpy(np.ascontiguousarray(ci, np.int32)).pin_memory()
    got = ni.count_host(h_rp, h_ci)
    torch.cuda.synchronize()
    ni.check()
    assert_same(got.numpy(), gpu_count(ni, rp, ci), name)
    assert_same(got.numpy(), oracle.count(rp, ci), name + " vs oracle")


def test_host_entry_rejects_unpinned_tensors(ni):
    rp, ci = gg.er(100, 0.1, 2)
    with pytest.raises(ValueError):
        ni.count_host(torch.from_numpy(rp), torch.from_numpy(ci))


def _with_isolated(rp, ci, extra):
    rp = np.concatenate([rp, np.full(extra, rp[-1], dtype=rp.dtype)])
    return rp, ci


def test_four_cycle_team_tier_both_modes(ni):
    # roots with more than 12288 wedges count in a dense row shared by a
    # cluster of CTAs: K3,9000 (W = 18000 against u ~ 9000) reads the row
    # back by sweeps; K2,13000 with 200000 isolated vertices (W = 13000,
    # u ~ 213000) marks first visitors per wedge
    a, b = 3, 9000
    assert_same(gpu_count(ni, *gg.complete_bipartite(a, b)), closed_complete_bipartite(a, b), "K3,9000")
    a, b, extra = 2, 13000, 200000
    rp, ci = _with_isolated(*gg.complete_bipartite(a, b), extra)
    exp = np.concatenate([closed_complete_bipartite(a, b), np.zeros((extra, 15), np.int64)])
    assert_same(gpu_count(ni, rp, ci), exp, "K2,13000 + isolated")


def test_empty_and_edgeless(ni):
    rp = np.zeros(6, np.int32)
    assert_same(gpu_count(ni, rp, np.zeros(0, np.int32)), np.zeros((5, 15), np.int64), "edgeless")
    out = ni.count(torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert out.shape == (0, 15)


def test_er2000_full_vs_oracle_and_definition(ni):
    rp, ci = gg.er(2000, 0.01, 1)
    got = gpu_count(ni, rp, ci)
    assert_same(got, oracle.count(rp, ci), "ER2000 vs three-stage oracle")
    assert_same(got, oracle.definition_count(rp, ci), "ER2000 vs definition")


@pytest.mark.parametrize("name,make", [
    ("rmat12", lambda: gg.rmat(12, 16, seed=3)),
    ("rmat14", lambda: gg.rmat(14, 16, seed=4)),
    ("chunglu20k", lambda: gg.chunglu(20000, 2.2, 12.0, 5)),
    ("er_dense", lambda: gg.er(600, 0.5, 6)),
    ("er_sparse", lambda: gg.er_mean_degree(50000, 6, 7)),
])
def test_medium_graphs_full_vs_oracle(ni, name, make):
    rp, ci = make()
    assert_same(gpu_count(ni, rp, ci), oracle.count(rp, ci), name)


def test_repeated_calls_identical(ni):
    rp, ci = gg.rmat(13, 16, seed=8)
    a = gpu_count(ni, rp, ci)
    for _ in range(3):
        assert np.array_equal(gpu_count(ni, rp, ci), a)


def test_batch_equals_single(ni):
    graphs = [gg.chunglu(int(n), 2.5, 8.0, 100 + i) for i, n in enumerate([50, 3, 1, 700, 2500, 90, 1200])]
    graphs.append(gg.complete(30))
    graphs.append(gg.complete_bipartite(3, 9000))                    # a root of the 4-cycle team tier
    graphs.append((np.zeros(4, np.int32), np.zeros(0, np.int32)))   # edgeless graph of 3 vertices
    rowptr, colidx, vo, eo = gg.pack(graphs)
    dev = torch.device("cuda:0")
    out = ni.count_batch(torch.from_numpy(rowptr.astype(np.int32)).to(dev), torch.from_numpy(colidx).to(dev),
                         torch.from_numpy(vo).to(dev), torch.from_numpy(eo).to(dev))
    ni.check()
    got = out.cpu().numpy()
    for g, (rp, ci) in enumerate(graphs):
        rows = got[vo[g]:vo[g + 1]]
        assert_same(rows, oracle.count(rp, ci), f"graph {g} in batch")
        assert_same(rows, gpu_count(ni, rp, ci), f"graph {g} batch vs alone")


def _expect_status(ni, rp, ci, status):
    dev = torch.device("cuda:0")
    ni.last_status()   # clear
    ni.count(torch.as_tensor(rp, dtype=torch.int32, device=dev), torch.as_tensor(ci, dtype=torch.int32, device=dev))
    assert ni.last_status() == status


def test_device_detected_errors(ni):
    from paper_2606_29651_gb300 import Status
    # rowptr[n] != m, out-of-range column, self-loop, unsorted row
    _expect_status(ni, [0, 1, 2], [1, 0, 0], Status.EINVAL)
    _expect_status(ni, [0, 1, 2], [7, 0], Status.EINVAL)
    _expect_status(ni, [0, 2, 3], [0, 1, 0], Status.ENOTSIMPLE)
    _expect_status(ni, [0, 2, 3, 4], [2, 1, 0, 0], Status.ENOTSIMPLE)
    # a clean graph after errors reports OK again
    _expect_status(ni, *gg.complete(5), Status.OK)


def test_validate_detects_asymmetry(ni):
    from paper_2606_29651_gb300 import Status
    dev = torch.device("cuda:0")
    ni.last_status()
    rp = torch.tensor([0, 1, 1], dtype=torch.int32, device=dev)     # 0 -> 1 without 1 -> 0
    ci = torch.tensor([1], dtype=torch.int32, device=dev)
    ni.validate(rp, ci)
    assert ni.last_status() == Status.ENOTSIMPLE
    rp2, ci2 = gg.rmat(10, 8, seed=1)
    ni.validate(torch.from_numpy(rp2).to(dev), torch.from_numpy(ci2).to(dev))
    assert ni.last_status() == Status.OK


@pytest.mark.parametrize("name,make", [
    ("er400", lambda: gg.er(400, 0.06, 41)),
    ("rmat10", lambda: gg.rmat(10, 16, seed=42)),
    ("dense80", lambda: gg.er(80, 0.6, 43)),
    ("k30", lambda: gg.complete(30)),
])
def test_induced_counts_vs_definition(ni, name, make):
    rp, ci = make()
    dev = torch.device("cuda:0")
    out = ni.count_induced(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev))
    ni.check()
    assert_same(out.cpu().numpy(), oracle.induced_count(rp, ci), name)


def test_degree_above_bound_stops_with_eoverflow(ni):
    # A star with 2^20 + 1 leaves: its centre's degree is above the bound
    # under which every count and intermediate fits int64, so the degree pass
    # records EOVERFLOW and every later stage returns without running.
    from paper_2606_29651_gb300 import Status
    k = (1 << 20) + 1
    rp = np.zeros(k + 2, np.int64)
    rp[1] = k
    rp[2:] = k + np.arange(1, k + 1)
    ci = np.concatenate([np.arange(1, k + 1), np.zeros(k, np.int64)]).astype(np.int32)
    _expect_status(ni, rp.astype(np.int32), ci, Status.EOVERFLOW)
    # exactly at the bound it counts, and the same stream reports OK again
    k = 1 << 20
    rp = np.zeros(k + 2, np.int64)
    rp[1] = k
    rp[2:] = k + np.arange(1, k + 1)
    ci = np.concatenate([np.arange(1, k + 1), np.zeros(k, np.int64)]).astype(np.int32)
    got = gpu_count(ni, rp.astype(np.int32), ci)
    exp_centre = [k, 0, k * (k - 1) // 2, 0, 0, 0, 0, k * (k - 1) * (k - 2) // 6, 0, 0, 0, 0, 0, 0, 0]
    assert got[0].tolist() == exp_centre
    assert got[1].tolist() == [1, k - 1, 0, 0, 0, 0, (k - 1) * (k - 2) // 2, 0, 0, 0, 0, 0, 0, 0, 0]
    assert (got[2:] == got[1]).all()


@pytest.fixture
def tuning(ni):
    saved = ni.get_tuning()
    yield ni
    ni.set_tuning(**saved)


@pytest.mark.parametrize("name,make", [
    ("er_dense", lambda: gg.er(600, 0.5, 6)),
    ("rmat14", lambda: gg.rmat(14, 16, seed=4)),
    ("chunglu20k", lambda: gg.chunglu(20000, 2.2, 12.0, 5)),
])
def test_cta_tier_paths_at_low_thresholds(tuning, name, make):
    # With low routing limits the CTA tiers of the triangle and aggregate
    # stages meet roots of every kind on small graphs: bit matrix (out-degree
    # <= 24), shared hash without the bit matrix (<= 48), and binary searches
    # of N+(u) with a K4 enumeration per triangle beyond.
    rp, ci = make()
    exp = oracle.count(rp, ci)
    tuning.set_tuning(warp_maxd=4, tri_bits_maxd=24, tri_hash_maxd=48)
    assert_same(gpu_count(tuning, rp, ci), exp, name + " low limits")
    tuning.set_tuning(warp_maxd=2, tri_bits_maxd=2, tri_hash_maxd=2)
    assert_same(gpu_count(tuning, rp, ci), exp, name + " binary searches only")


@pytest.mark.parametrize("name,make", [
    ("rmat12", lambda: gg.rmat(12, 16, seed=3)),
    ("er_dense", lambda: gg.er(600, 0.5, 6)),
    ("chunglu20k", lambda: gg.chunglu(20000, 2.2, 12.0, 5)),
    ("k3_900", lambda: gg.complete_bipartite(3, 900)),
])
def test_key_tiled_four_cycle_tier_for_every_root(tuning, name, make):
    # Every root with more than two wedges goes to the widest 4-cycle tier.
    rp, ci = make()
    exp = oracle.count(rp, ci)
    tuning.set_tuning(c4_warp_maxw=2, c4_team_minw=2)
    assert_same(gpu_count(tuning, rp, ci), exp, name + " all roots in the widest tier")
    tuning.set_tuning(c4_warp_maxw=300, c4_team_minw=600)
    assert_same(gpu_count(tuning, rp, ci), exp, name + " mixed tiers")

"""Full-size parity on the large configurations, element by element.

  * ER n = 1e6, mean degree 32 (the headline graph): every one of the
    15 x 10^6 entries against the three-stage oracle.
  * R-MAT scale 22: every row against invariants that hold at any size, and
    sampled rows against the oracle's per-vertex mode, chosen so that every
    tier kernel's roots are among them (the CTA and 1024-thread triangle and
    aggregate tiers, every 4-cycle tier up to the key-tiled one), plus
    vertices of degree 300-5000, random low-degree vertices and neighbours of
    the largest hub. The per-vertex oracle costs about d_x^2 plus, for every
    neighbour y, the intersections of y's row with its neighbours' rows; a
    vertex next to a hub of degree ~1.6e5 can take hours, so each tier
    contributes its cheapest roots under a per-vertex bound (about 20 s of
    one core) and a few random ones under that bound.
  * The batched configuration at its full 8192 Chung-Lu graphs: every graph
    of the one batched call against the oracle.
  * A served stream of 120 requests of up to 1e5 edges: every result
    against the oracle.
Kept in a file of its own so that it runs after the smaller GPU tests."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import cheap_sum_checks
from test_gpu_parity import assert_same, gpu_count

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VERTEX_COST_CAP = 3e9   # oracle work units of one sampled vertex (~1.5e8 per second per core)


@pytest.fixture(scope="module")
def ni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_29651_gb300 as ni
    ni.build()
    return ni


def test_er_1e6_every_row(ni):
    rp, ci = gg.er_mean_degree(1_000_000, 32, 1)
    got = gpu_count(ni, rp, ci)
    assert cheap_sum_checks(rp, got) == []
    assert_same(got, oracle.count(rp, ci), "ER n=1e6, all rows")


def oracle_cost(rp, ci):
    """Work of the per-vertex oracle for every vertex x (model):
    d_x^2 + sum over y in N(x) of sum over z in N(y) of min(d_y, d_z)."""
    n = len(rp) - 1
    d = np.diff(rp).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    s_y = np.bincount(src, weights=np.minimum(d[src], d[ci]), minlength=n)
    return d.astype(np.float64) ** 2 + np.bincount(src, weights=s_y[ci], minlength=n)


def tier_sample(rp, ci, seed):
    import bench
    rng = np.random.default_rng(seed)
    d = np.diff(rp)
    cost = oracle_cost(rp, ci)
    tiers = bench.vertex_tiers(rp, ci)
    pick, per_tier = set(), {}

    def take(name, cand, cheapest, rand):
        cand = cand[cost[cand] <= VERTEX_COST_CAP]
        if len(cand) == 0:
            per_tier[name] = 0
            return
        by_cost = cand[np.argsort(cost[cand], kind="stable")]
        chosen = set(int(v) for v in by_cost[:cheapest])
        rest = np.array(sorted(set(cand.tolist()) - chosen), dtype=np.int64)
        if len(rest) and rand:
            chosen.update(int(v) for v in rng.choice(rest, size=min(rand, len(rest)), replace=False))
        per_tier[name] = len(chosen)
        pick.update(chosen)

    for name, cheapest, rand in (("k_tri_cta", 6, 4), ("k_tri_big", 5, 0), ("big_hash", 2, 0),
                                 ("big_search", 2, 0), ("k_c4_warp_big", 2, 2), ("k_c4_midp", 2, 2),
                                 ("k_c4_mid", 2, 2), ("k_c4_cta", 2, 2), ("k_c4_tiled", 8, 0)):
        take(name, np.asarray(tiers[name], dtype=np.int64), cheapest, rand)
    take("degree 300-5000", np.flatnonzero((d >= 300) & (d <= 5000)), 0, 6)
    take("degree 1-64", np.flatnonzero((d >= 1) & (d <= 64)), 0, 100)
    top = int(np.argmax(d))
    nb = ci[rp[top]:rp[top + 1]].astype(np.int64)
    take("neighbours of the largest hub", nb[d[nb] <= 64], 10, 10)
    return np.array(sorted(pick), dtype=np.int32), per_tier, cost


def test_rmat22_rows_of_every_tier(ni):
    rp, ci = gg.rmat(22, 16, seed=1)
    got = gpu_count(ni, rp, ci)
    assert cheap_sum_checks(rp, got) == []
    verts, per_tier, cost = tier_sample(rp, ci, 12)
    for name in ("k_tri_cta", "k_tri_big", "k_c4_mid", "k_c4_cta", "k_c4_tiled"):
        assert per_tier[name] > 0, (name, per_tier)
    assert cost[verts].sum() < 1.5e11
    assert_same(got[verts], oracle.count_vertices(rp, ci, verts), f"sampled rows {per_tier}")


def test_batched_8192_graphs_every_graph(ni):
    graphs = gg.chunglu_batch(8192, 2.5, 8.0, 50, 5000, seed=1)
    rowptr, colidx, vo, eo = gg.pack(graphs)
    dev = torch.device("cuda:0")
    out = ni.count_batch(torch.from_numpy(rowptr.astype(np.int32)).to(dev), torch.from_numpy(colidx).to(dev),
                         torch.from_numpy(vo).to(dev), torch.from_numpy(eo).to(dev))
    ni.check()
    got = out.cpu().numpy()
    for g, (rp, ci) in enumerate(graphs):
        assert_same(got[vo[g]:vo[g + 1]], oracle.count(rp, ci), f"graph {g} of 8192")


def test_served_stream_every_result(ni):
    from paper_2606_29651_gb300.serve import Server
    nreq = 120
    u = gg.uniform(7, 11, 4 * nreq)
    graphs = []
    for i in range(nreq):
        e = float(np.exp(np.log(1e3) + u[i] * (np.log(1e5) - np.log(1e3))))
        dmean = 4 + 28 * u[nreq + i]
        n = max(int(2 * e / dmean), 8)
        if u[2 * nreq + i] < 0.5:
            graphs.append(gg.er_mean_degree(n, dmean, 500 + i))
        else:
            graphs.append(gg.chunglu(n, 2.2 + 0.8 * u[3 * nreq + i], dmean, 500 + i))
    with Server(0, mem_budget=2 << 30, streams=3, max_batch_graphs=32) as srv:
        futs = [srv.submit(rp, ci) for rp, ci in graphs]
        res = [f.result(timeout=600) for f in futs]
        assert srv.batches < nreq
    for i, (rp, ci) in enumerate(graphs):
        assert_same(res[i], oracle.count(rp, ci), f"request {i}")

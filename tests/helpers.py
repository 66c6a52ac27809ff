"""Shared test helpers: closed forms and independent graphlet totals.

Nothing here calls the library or the oracle; these are the pins the oracle
(and, through it, the CUDA path) is checked against.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np


def closed_complete(n: int) -> list:
    """Orbit row of every vertex of K_n (all vertices alike), m = n - 1."""
    m = n - 1
    c2 = lambda a: comb(a, 2) if a >= 0 else 0  # noqa: E731
    c3 = lambda a: comb(a, 3) if a >= 0 else 0  # noqa: E731
    return [m, m * (m - 1), c2(m), c2(m), m * (m - 1) * (m - 2), m * (m - 1) * (m - 2),
            m * c2(m - 1), c3(m), 3 * c3(m), m * c2(m - 1), m * (m - 1) * (m - 2),
            c2(m) * (m - 2), c2(m) * (m - 2), m * c2(m - 1), c3(m)]


def closed_star(k: int) -> np.ndarray:
    """Rows of the star with centre 0 and leaves 1..k."""
    out = np.zeros((k + 1, 15), dtype=np.int64)
    out[0, 0], out[0, 2], out[0, 7] = k, comb(k, 2), comb(k, 3)
    for i in range(1, k + 1):
        out[i, 0], out[i, 1], out[i, 6] = 1, k - 1, comb(k - 1, 2)
    return out


def closed_cycle(n: int) -> np.ndarray:
    row = [2, 2, 1, 0] + [0] * 11
    if n == 3:
        row[3] = 1
    if n >= 4:
        row[4], row[5] = 2, 2
    if n == 4:
        row[8] = 1
    return np.tile(np.array(row, dtype=np.int64), (n, 1))


def closed_path(n: int) -> np.ndarray:
    out = np.zeros((n, 15), dtype=np.int64)
    for v in range(n):
        d = (v > 0) + (v < n - 1)
        out[v, 0] = d
        out[v, 1] = (v - 2 >= 0) + (v + 2 <= n - 1)
        out[v, 2] = comb(d, 2)
        out[v, 4] = (v - 3 >= 0) + (v + 3 <= n - 1)
        # windows of 4 consecutive vertices with v at position 1 or 2
        out[v, 5] = sum(1 for s in (v - 1, v - 2) if s >= 0 and s + 3 <= n - 1)
    return out


def closed_complete_bipartite(a: int, b: int) -> np.ndarray:
    """Rows of K_{a,b}: side A = 0..a-1 (degree b), side B = a..a+b-1."""
    def side(a_, b_):
        r = [0] * 15
        r[0], r[1], r[2] = b_, b_ * (a_ - 1), comb(b_, 2)
        r[4] = b_ * (a_ - 1) * (b_ - 1)
        r[5] = b_ * (b_ - 1) * (a_ - 1)
        r[6] = b_ * comb(a_ - 1, 2) if a_ >= 1 else 0
        r[7] = comb(b_, 3)
        r[8] = (a_ - 1) * comb(b_, 2) if a_ >= 1 else 0
        return r
    rows = [side(a, b)] * a + [side(b, a)] * b
    return np.array(rows, dtype=np.int64)


def graphlet_totals(rowptr, colidx) -> dict:
    """Number of (non-induced) copies of each connected graphlet, by formulas
    independent of the orbit machinery: scipy sparse products and networkx
    clique enumeration."""
    import networkx as nx
    import scipy.sparse as sp

    n = len(rowptr) - 1
    d = np.diff(rowptr).astype(np.int64)
    rows = np.repeat(np.arange(n), d)
    A = sp.csr_matrix((np.ones(len(colidx), dtype=np.int64), (rows, colidx)), shape=(n, n))
    A2 = (A @ A).tocsr()
    t_edge = A2.multiply(A).tocsr()                 # t_uv on every (u, v) in E
    tri_at = np.asarray(t_edge.sum(axis=1)).ravel() // 2
    ntri = int(tri_at.sum() // 3)
    up = sp.triu(t_edge, k=1).tocoo()
    eu, ev = np.nonzero(sp.triu(A, k=1))
    p3 = int(sum(comb(int(x), 2) for x in d))
    p4 = int(((d[eu] - 1) * (d[ev] - 1)).sum()) - 3 * ntri
    s3 = int(sum(comb(int(x), 3) for x in d))
    offd = sp.triu(A2, k=1).tocoo()
    c4 = int(sum(comb(int(c), 2) for c in offd.data)) // 2
    paw = int((tri_at * (d - 2)).sum())
    diamond = int(sum(comb(int(c), 2) for c in up.data))
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(zip(eu.tolist(), ev.tolist()))
    k4 = 0
    for c in nx.enumerate_all_cliques(G):
        if len(c) == 4:
            k4 += 1
        elif len(c) > 4:
            break
    return dict(edge=len(colidx) // 2, p3=p3, tri=ntri, p4=p4, star=s3, c4=c4, paw=paw,
                diamond=diamond, k4=k4)


def orbit_sums_expected(tot: dict) -> np.ndarray:
    """Per-orbit sums over all vertices = graphlet count x orbit size."""
    return np.array([2 * tot["edge"], 2 * tot["p3"], tot["p3"], 3 * tot["tri"], 2 * tot["p4"],
                     2 * tot["p4"], 3 * tot["star"], tot["star"], 4 * tot["c4"], tot["paw"],
                     2 * tot["paw"], tot["paw"], 2 * tot["diamond"], 2 * tot["diamond"],
                     4 * tot["k4"]], dtype=np.int64)


def cheap_sum_checks(rowptr, psi) -> list:
    """Invariants that hold at any size and need only degrees: returns the
    list of violated checks (empty when all hold)."""
    d = np.diff(np.asarray(rowptr)).astype(np.int64)
    s = psi.sum(axis=0)
    bad = []
    checks = {
        "psi0 = 2|E|": s[0] == d.sum(),
        "psi0 = deg": np.array_equal(psi[:, 0], d),
        "sum psi1 = 2 sum psi2": s[1] == 2 * s[2],
        "psi2 = C(d,2)": np.array_equal(psi[:, 2], d * (d - 1) // 2),
        "psi7 = C(d,3)": np.array_equal(psi[:, 7], d * (d - 1) * (d - 2) // 6),
        "sum psi3 = 0 mod 3": s[3] % 3 == 0,
        "sum psi4 = sum psi5": s[4] == s[5],
        "sum psi6 = 3 sum psi7": s[6] == 3 * s[7],
        "sum psi8 = 0 mod 4": s[8] % 4 == 0,
        "sum psi10 = 2 sum psi9": s[10] == 2 * s[9],
        "sum psi9 = sum psi11": s[9] == s[11],
        "sum psi12 = sum psi13": s[12] == s[13],
        "sum psi12 even": s[12] % 2 == 0,
        "sum psi14 = 0 mod 4": s[14] % 4 == 0,
        "nonnegative": bool((psi >= 0).all()),
    }
    for k, ok in checks.items():
        if not ok:
            bad.append(k)
    return bad


def random_small_graphs(count: int, nmax: int, seed: int):
    """Seeded random graphs with n <= nmax as (n, edge list)."""
    import random
    rng = random.Random(seed)
    out = []
    for _ in range(count):
        n = rng.randint(1, nmax)
        p = rng.random()
        out.append((n, [(u, v) for u, v in itertools.combinations(range(n), 2) if rng.random() < p]))
    return out


def read_golden(path: str):
    """Parse tests/golden/hand_worked.txt into [(name, n, edges, table)]."""
    graphs, cur = [], None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "graph":
                cur = [tok[1], int(tok[2]), [], {}]
                graphs.append(cur)
            elif tok[0] == "edges":
                cur[2] = [tuple(int(x) for x in e.split("-")) for e in tok[1:]]
            else:
                cur[3][int(tok[0])] = [int(x) for x in tok[1:]]
    res = []
    for name, n, edges, rows in graphs:
        tab = np.array([rows[v] for v in range(n)], dtype=np.int64)
        res.append((name, n, edges, tab))
    return res

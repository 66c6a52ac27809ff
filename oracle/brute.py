"""ORACLE (test infrastructure): brute-force non-induced orbit counts.

The definitions of Sec. 3 (Defs. 1-5) written out with no cleverness at all,
for graphs of a dozen vertices at most: every vertex subset V' of size 2, 3
or 4, every subset E' of the edges of G inside V', kept when (V', E') is
connected; the graphlet is recognised by its edge count and degree sequence
and every vertex is credited with its orbit (numbering as in oracle/enumerate.c:
0 edge, 1-2 path P3 end/middle, 3 triangle, 4-5 path P4 end/interior,
6-7 3-star leaf/centre, 8 4-cycle, 9-11 paw by degree 1/2/3, 12-13 diamond
by degree 2/3, 14 K4).

Only tests/ may import this module.
"""
from __future__ import annotations

import itertools


def _connected(vertices, edges) -> bool:
    adj = {v: set() for v in vertices}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    start = vertices[0]
    seen = {start}
    stack = [start]
    while stack:
        c = stack.pop()
        for w in adj[c]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == len(vertices)


def _orbit(k: int, nedges: int, degs: dict, v) -> int:
    d = degs[v]
    ds = sorted(degs.values())
    if k == 2:
        return 0
    if k == 3:
        return 3 if nedges == 3 else (1 if d == 1 else 2)
    if nedges == 3:                      # trees on 4 vertices
        if ds[-1] == 3:                  # 3-star
            return 7 if d == 3 else 6
        return 4 if d == 1 else 5        # path P4
    if nedges == 4:
        if ds == [2, 2, 2, 2]:           # 4-cycle
            return 8
        return {1: 9, 2: 10, 3: 11}[d]   # paw (tailed triangle)
    if nedges == 5:                      # diamond
        return 12 if d == 2 else 13
    return 14                            # K4


def brute_count(n: int, edges, induced: bool = False) -> list:
    """psi[x][k] for every vertex x of the simple graph (range(n), edges).

    With induced=True only E' = all edges inside V' is counted (Def. 2)."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    psi = [[0] * 15 for _ in range(n)]
    for k in (2, 3, 4):
        for vs in itertools.combinations(range(n), k):
            inside = [(a, b) for a, b in itertools.combinations(vs, 2) if b in adj[a]]
            sizes = [len(inside)] if induced else range(k - 1, len(inside) + 1)
            for r in sizes:
                for sub in itertools.combinations(inside, r):
                    if not _connected(list(vs), sub):
                        continue
                    degs = {v: 0 for v in vs}
                    for a, b in sub:
                        degs[a] += 1
                        degs[b] += 1
                    for v in vs:
                        psi[v][_orbit(k, r, degs, v)] += 1
    return psi

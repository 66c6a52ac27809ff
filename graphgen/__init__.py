"""Seeded synthetic graph generators (inputs only; no orbit arithmetic).

Both the CPU oracle and the CUDA path are fed from here, so that they see
identical graphs. Every generator returns a simple undirected graph as CSR
``(rowptr int32[n+1], colidx int32[m])`` with ``m = 2|E|`` and every row sorted
ascending: the input contract of the library.

The C implementation lives in ``graphgen.c`` and is compiled on first use
with the host C compiler (``gcc``), into this directory.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into _graphgen.so (host code, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
                   _SRC, "-o", tmp, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    vp = ctypes.c_void_p
    lib.gg_er.restype = vp
    lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64]
    lib.gg_rmat.restype = vp
    lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_uint64]
    lib.gg_chunglu.restype = vp
    lib.gg_chunglu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64]
    lib.gg_from_edges.restype = vp
    lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp]
    lib.gg_n.restype = ctypes.c_int32
    lib.gg_n.argtypes = [vp]
    lib.gg_m.restype = ctypes.c_int64
    lib.gg_m.argtypes = [vp]
    lib.gg_copy_out.restype = None
    lib.gg_copy_out.argtypes = [vp, vp, vp]
    lib.gg_free.restype = None
    lib.gg_free.argtypes = [vp]
    lib.gg_uniform.restype = None
    lib.gg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, vp]
    _lib = lib
    return lib


def _take(handle):
    lib = _load()
    if not handle:
        raise ValueError("graph generation failed (bad arguments or out of memory)")
    try:
        n = lib.gg_n(handle)
        m = lib.gg_m(handle)
        rowptr = np.empty(n + 1, dtype=np.int32)
        colidx = np.empty(max(m, 0), dtype=np.int32)
        lib.gg_copy_out(handle, rowptr.ctypes.data, colidx.ctypes.data if m else None)
    finally:
        lib.gg_free(handle)
    return rowptr, colidx


def er(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p), each pair independently with probability p."""
    return _take(_load().gg_er(int(n), float(p), int(seed) & (2**64 - 1)))


def er_mean_degree(n: int, dmean: float, seed: int):
    """G(n, p) with p = dmean / (n - 1)."""
    p = dmean / max(n - 1, 1)
    return er(n, p, seed)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """R-MAT graph on 2^scale vertices; loops and duplicates removed, symmetrised."""
    return _take(_load().gg_rmat(int(scale), int(edge_factor), float(a), float(b), float(c),
                                 int(seed) & (2**64 - 1)))


def chunglu(n: int, gamma: float = 2.5, dmean: float = 8.0, seed: int = 1):
    """Erased Chung-Lu graph with power-law weights of exponent gamma."""
    return _take(_load().gg_chunglu(int(n), float(gamma), float(dmean), int(seed) & (2**64 - 1)))


def from_edges(n: int, edges):
    """CSR of an explicit undirected edge list [(u, v), ...] (loops/duplicates dropped)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    eu = np.ascontiguousarray(e[:, 0], dtype=np.int32)
    ev = np.ascontiguousarray(e[:, 1], dtype=np.int32)
    h = _load().gg_from_edges(int(n), int(len(e)), eu.ctypes.data if len(e) else None,
                              ev.ctypes.data if len(e) else None)
    return _take(h)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Seeded uniform doubles in [0, 1) (xoshiro256** stream `stream`)."""
    out = np.empty(int(count), dtype=np.float64)
    if count:
        _load().gg_uniform(int(seed) & (2**64 - 1), int(stream) & (2**64 - 1), int(count),
                           out.ctypes.data)
    return out


# ---------------------------------------------------------------- named graphs

def complete(n: int):
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def star(k: int):
    """Centre 0 with k leaves 1..k."""
    return from_edges(k + 1, [(0, i) for i in range(1, k + 1)])


def path(n: int):
    return from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int):
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def complete_bipartite(a: int, b: int):
    """Side A = 0..a-1, side B = a..a+b-1."""
    return from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def batch_sizes(count: int, lo: int = 50, hi: int = 5000, seed: int = 1) -> np.ndarray:
    """Vertex counts floor(exp(U[ln lo, ln hi])) for a batch of graphs."""
    u = uniform(seed, 7, count)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def chunglu_batch(count: int, gamma: float = 2.5, dmean: float = 8.0, lo: int = 50,
                  hi: int = 5000, seed: int = 1):
    """A batch of Chung-Lu graphs of log-uniform size; returns a list of CSR tuples."""
    sizes = batch_sizes(count, lo, hi, seed)
    return [chunglu(int(n), gamma, dmean, seed * 1_000_003 + i) for i, n in enumerate(sizes)]


def pack(graphs):
    """Pack CSR graphs (local ids) into the batched layout.

    Returns (rowptr, colidx, vtx_offset, edge_offset): rowptr concatenates each
    graph's local rowptr[0..n_g-1] shifted by edge_offset[g] plus a final
    entry, colidx concatenates local column ids, vtx_offset/edge_offset are
    int64 prefix sums of n_g and m_g.
    """
    ns = np.array([len(r) - 1 for r, _ in graphs], dtype=np.int64)
    ms = np.array([len(c) for _, c in graphs], dtype=np.int64)
    vo = np.zeros(len(graphs) + 1, dtype=np.int64)
    eo = np.zeros(len(graphs) + 1, dtype=np.int64)
    vo[1:] = np.cumsum(ns)
    eo[1:] = np.cumsum(ms)
    rowptr = np.empty(int(vo[-1]) + 1, dtype=np.int64)
    for g, (r, _) in enumerate(graphs):
        rowptr[vo[g]:vo[g + 1]] = r[:-1].astype(np.int64) + eo[g]
    rowptr[-1] = eo[-1]
    colidx = np.concatenate([c for _, c in graphs]) if len(graphs) else np.zeros(0, np.int32)
    return rowptr, colidx.astype(np.int32), vo, eo

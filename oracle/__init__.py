"""ORACLE -- test infrastructure, not the product.

Plain, slow CPU implementations of what the library computes: per-vertex
counts of the 15 non-induced graphlet orbits on up to four vertices
(Sec. 3, Defs. 1-5).

  * ``count`` / ``count_vertices``: the paper's method as printed, in plain C
    (``niorca_oracle.c``): Stage I per-edge triangles (Algorithm 1),
    Stage II ``CountK4`` (Algorithm 2), Stage III the f* variables of Table 1
    and the equations of Sec. 5 and the Appendix.
  * ``definition_count`` / ``definition_count_vertices``: the definition
    written out (``enumerate.c``): every connected vertex set of size 2-4 and
    every connected spanning edge subset, classified.
  * ``brute_count`` (``brute.py``): the definition over all vertex subsets in
    pure Python, for graphs of about a dozen vertices.
  * ``induced_count``: induced orbit counts (Def. 2: E' = every edge inside
    V'), by the same enumeration.

Every function here is pinned by the tests (closed forms, invariants, brute
force). Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package; the
library itself never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .brute import brute_count  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "niorca_oracle.c"), os.path.join(_HERE, "enumerate.c")]
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

# reading switches and error codes of niorca_oracle.c
READ_F69_EYZ = 1
READ_NEIGH_NO_RESET = 2
READ_FIG3B_ORDERED = 4
N_MUTATIONS = 12


def build(force: bool = False) -> str:
    """Compile the C oracle into _oracle.so (host code, OpenMP)."""
    with _lock:
        newest = max(os.path.getmtime(s) for s in _SRCS)
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < newest
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", *_SRCS, "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.orc_count.restype = ctypes.c_int
    lib.orc_count.argtypes = [i32, vp, vp, vp, ctypes.c_int, ctypes.c_int]
    lib.orc_count_vertices.restype = ctypes.c_int
    lib.orc_count_vertices.argtypes = [i32, vp, vp, i32, vp, vp, ctypes.c_int, ctypes.c_int]
    lib.orc_stage1.restype = None
    lib.orc_stage1.argtypes = [i32, vp, vp, vp]
    lib.orc_stage2.restype = ctypes.c_int
    lib.orc_stage2.argtypes = [i32, vp, vp, vp, ctypes.c_int]
    lib.orc_set_threads.restype = None
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_max_threads.restype = ctypes.c_int
    lib.orc_max_threads.argtypes = []
    lib.def_count.restype = None
    lib.def_count.argtypes = [i32, vp, vp, vp]
    lib.def_count_induced.restype = None
    lib.def_count_induced.argtypes = [i32, vp, vp, vp]
    lib.def_count_vertices.restype = None
    lib.def_count_vertices.argtypes = [i32, vp, vp, i32, vp, vp]
    _lib = lib
    return lib


def _csr(rowptr, colidx):
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    if len(ci) == 0:
        ci = np.zeros(1, dtype=np.int32)
    return len(rp) - 1, rp, ci


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def count(rowptr, colidx, flags: int = 0, mutation: int = 0) -> np.ndarray:
    """Orbit counts of every vertex by the paper's three stages; int64[n, 15]."""
    n, rp, ci = _csr(rowptr, colidx)
    out = np.zeros((max(n, 1), 15), dtype=np.int64)
    err = _load().orc_count(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data, int(flags), int(mutation))
    if err:
        raise RuntimeError(f"oracle error {err}")
    return out[:n]


def count_vertices(rowptr, colidx, verts, flags: int = 0, mutation: int = 0) -> np.ndarray:
    """Orbit counts of the listed vertices only (Stage III per vertex); int64[len(verts), 15]."""
    n, rp, ci = _csr(rowptr, colidx)
    v = np.ascontiguousarray(verts, dtype=np.int32)
    out = np.zeros((max(len(v), 1), 15), dtype=np.int64)
    err = _load().orc_count_vertices(n, rp.ctypes.data, ci.ctypes.data, len(v), v.ctypes.data,
                                     out.ctypes.data, int(flags), int(mutation))
    if err:
        raise RuntimeError(f"oracle error {err}")
    return out[:len(v)]


def stage1_triangles(rowptr, colidx) -> np.ndarray:
    """Stage I: triangle count of the edge at every CSR position; int32[m]."""
    n, rp, ci = _csr(rowptr, colidx)
    tri = np.zeros(max(len(colidx), 1), dtype=np.int32)
    _load().orc_stage1(n, rp.ctypes.data, ci.ctypes.data, tri.ctypes.data)
    return tri[:len(colidx)]


def stage2_k4(rowptr, colidx, flags: int = 0) -> np.ndarray:
    """Stage II: number of K4 containing each vertex; int64[n]."""
    n, rp, ci = _csr(rowptr, colidx)
    k4 = np.zeros(max(n, 1), dtype=np.int64)
    err = _load().orc_stage2(n, rp.ctypes.data, ci.ctypes.data, k4.ctypes.data, int(flags))
    if err:
        raise RuntimeError(f"oracle error {err}")
    return k4[:n]


def definition_count(rowptr, colidx) -> np.ndarray:
    """Orbit counts of every vertex by enumerating subgraphs (the definition); int64[n, 15]."""
    n, rp, ci = _csr(rowptr, colidx)
    out = np.zeros((max(n, 1), 15), dtype=np.int64)
    _load().def_count(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data)
    return out[:n]


def definition_count_vertices(rowptr, colidx, verts) -> np.ndarray:
    """Enumeration-based orbit counts of the listed vertices; int64[len(verts), 15]."""
    n, rp, ci = _csr(rowptr, colidx)
    v = np.ascontiguousarray(verts, dtype=np.int32)
    out = np.zeros((max(len(v), 1), 15), dtype=np.int64)
    _load().def_count_vertices(n, rp.ctypes.data, ci.ctypes.data, len(v), v.ctypes.data, out.ctypes.data)
    return out[:len(v)]


def induced_count(rowptr, colidx) -> np.ndarray:
    """Induced orbit counts of every vertex by enumeration (Def. 2); int64[n, 15]."""
    n, rp, ci = _csr(rowptr, colidx)
    out = np.zeros((max(n, 1), 15), dtype=np.int64)
    _load().def_count_induced(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data)
    return out[:n]

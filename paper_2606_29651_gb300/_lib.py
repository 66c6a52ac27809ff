"""ctypes binding of libniorca.so (include/niorca.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the computation
runs in the library's CUDA kernels. There is no CPU fallback: if the shared
library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import enum
import os

import torch

from .builder import LIB


class Status(enum.IntEnum):
    OK = 0
    EINVAL = 1
    ENOTSIMPLE = 2
    EOVERFLOW = 3
    ENOMEM = 4
    ECUDA = 5
    ETIMEOUT = 6


class NiorcaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = Status(status)
        super().__init__(f"{where}: {self.status.name} ({_lib().niorca_status_string(int(status)).decode()})")


_handle = None


def _lib():
    global _handle
    if _handle is not None:
        return _handle
    if not os.path.exists(LIB):
        raise ImportError(f"libniorca.so is not built ({LIB}); run paper_2606_29651_gb300.build()")
    h = ctypes.CDLL(LIB)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    h.niorca_count.restype = ctypes.c_int
    h.niorca_count.argtypes = [vp, vp, i32, i64, vp, vp]
    h.niorca_count_induced.restype = ctypes.c_int
    h.niorca_count_induced.argtypes = [vp, vp, i32, i64, vp, vp]
    h.niorca_count_host.argtypes = [vp, vp, i32, i64, vp, vp]
    h.niorca_count_host.restype = ctypes.c_int
    h.niorca_count_batch.restype = ctypes.c_int
    h.niorca_count_batch.argtypes = [vp, vp, vp, vp, i32, i64, i64, vp, vp]
    h.niorca_validate.restype = ctypes.c_int
    h.niorca_validate.argtypes = [vp, vp, i32, i64, vp]
    h.niorca_last_status.restype = ctypes.c_int
    h.niorca_last_status.argtypes = [vp]
    h.niorca_workspace_bytes.restype = ctypes.c_size_t
    h.niorca_workspace_bytes.argtypes = [i32, i64]
    h.niorca_batch_workspace_bytes.restype = ctypes.c_size_t
    h.niorca_batch_workspace_bytes.argtypes = [i32, i64, i64]
    h.niorca_status_string.restype = ctypes.c_char_p
    h.niorca_status_string.argtypes = [ctypes.c_int]
    h.niorca_version.restype = i32
    h.niorca_version.argtypes = []
    h.niorca_profile_enable.restype = None
    h.niorca_profile_enable.argtypes = [i32]
    h.niorca_profile_read.restype = i32
    h.niorca_profile_read.argtypes = [vp, vp, i32]
    h.niorca_profile_reset.restype = None
    h.niorca_profile_reset.argtypes = []
    h.niorca_kernel_name.restype = ctypes.c_char_p
    h.niorca_kernel_name.argtypes = [i32]
    h.niorca_launch_count.restype = i64
    h.niorca_launch_count.argtypes = []
    h.niorca_set_tuning.restype = ctypes.c_int
    h.niorca_set_tuning.argtypes = [vp, i32]
    h.niorca_get_tuning.restype = i32
    h.niorca_get_tuning.argtypes = [vp, i32]
    _handle = h
    return h


def library():
    """The loaded ctypes handle (raises if the library is not built)."""
    return _lib()


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t: torch.Tensor):
    return t.data_ptr() if t.numel() else None


def count(rowptr: torch.Tensor, colidx: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """psi[v, k] for every vertex of the CSR graph (device int32 tensors).

    Enqueues on `stream` (default: torch's current stream) and returns the
    int64 [n, 15] output without synchronising.
    """
    _dev(rowptr, torch.int32, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    n = rowptr.numel() - 1
    if out is None:
        out = torch.empty((max(n, 0), 15), dtype=torch.int64, device=rowptr.device)
    _dev(out, torch.int64, "out")
    if out.numel() != 15 * max(n, 0):
        raise ValueError("out must hold n * 15 int64")
    st = _lib().niorca_count(_ptr(rowptr), _ptr(colidx), n, colidx.numel(), _ptr(out), _stream_ptr(stream))
    if st:
        raise NiorcaError(st, "niorca_count")
    return out


def _pinned(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if t.is_cuda or not t.is_pinned():
        raise ValueError(f"{name} must be a pinned (page-locked) CPU tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def count_host(rowptr: torch.Tensor, colidx: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """psi[v, k] for a CSR graph in pinned host memory, written into pinned
    host memory (niorca_count_host: the kernels read the CSR and write the
    counts across the host link, with no staging copy).

    Enqueues on `stream` (default: torch's current stream); `out` is valid
    once the stream has reached the end of the call.
    """
    _pinned(rowptr, torch.int32, "rowptr")
    _pinned(colidx, torch.int32, "colidx")
    n = rowptr.numel() - 1
    if out is None:
        out = torch.empty((max(n, 0), 15), dtype=torch.int64).pin_memory()
    _pinned(out, torch.int64, "out")
    if out.numel() != 15 * max(n, 0):
        raise ValueError("out must hold n * 15 int64")
    st = _lib().niorca_count_host(_ptr(rowptr), _ptr(colidx), n, colidx.numel(), _ptr(out), _stream_ptr(stream))
    if st:
        raise NiorcaError(st, "niorca_count_host")
    return out


def count_induced(rowptr: torch.Tensor, colidx: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Induced orbit counts psi'[v, k] (Def. 2), same conventions as count()."""
    _dev(rowptr, torch.int32, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    n = rowptr.numel() - 1
    if out is None:
        out = torch.empty((max(n, 0), 15), dtype=torch.int64, device=rowptr.device)
    _dev(out, torch.int64, "out")
    if out.numel() != 15 * max(n, 0):
        raise ValueError("out must hold n * 15 int64")
    st = _lib().niorca_count_induced(_ptr(rowptr), _ptr(colidx), n, colidx.numel(), _ptr(out),
                                     _stream_ptr(stream))
    if st:
        raise NiorcaError(st, "niorca_count_induced")
    return out


def count_batch(rowptr: torch.Tensor, colidx: torch.Tensor, vtx_offset: torch.Tensor, edge_offset: torch.Tensor,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Orbit counts of many packed graphs in one call (see niorca_count_batch)."""
    _dev(rowptr, torch.int32, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    _dev(vtx_offset, torch.int64, "vtx_offset")
    _dev(edge_offset, torch.int64, "edge_offset")
    g = vtx_offset.numel() - 1
    total_n = rowptr.numel() - 1
    if out is None:
        out = torch.empty((max(total_n, 0), 15), dtype=torch.int64, device=rowptr.device)
    _dev(out, torch.int64, "out")
    st = _lib().niorca_count_batch(_ptr(rowptr), _ptr(colidx), _ptr(vtx_offset), _ptr(edge_offset), g, total_n,
                                   colidx.numel(), _ptr(out), _stream_ptr(stream))
    if st:
        raise NiorcaError(st, "niorca_count_batch")
    return out


def validate(rowptr: torch.Tensor, colidx: torch.Tensor, stream=None) -> None:
    """Enqueue the full simple-graph check; read the verdict with last_status()."""
    _dev(rowptr, torch.int32, "rowptr")
    _dev(colidx, torch.int32, "colidx")
    st = _lib().niorca_validate(_ptr(rowptr), _ptr(colidx), rowptr.numel() - 1, colidx.numel(), _stream_ptr(stream))
    if st:
        raise NiorcaError(st, "niorca_validate")


def last_status(stream=None) -> Status:
    """Read and clear the status word of `stream` (default: torch's current
    stream) after the stream's work; errors of calls on other streams are
    not seen here."""
    return Status(_lib().niorca_last_status(_stream_ptr(stream)))


def check(stream=None) -> None:
    """Raise NiorcaError if a call on `stream` recorded a device-side error."""
    st = _lib().niorca_last_status(_stream_ptr(stream))
    if st:
        raise NiorcaError(st, "device status")


def workspace_bytes(n: int, m: int) -> int:
    return int(_lib().niorca_workspace_bytes(int(n), int(m)))


def batch_workspace_bytes(num_graphs: int, total_n: int, total_m: int) -> int:
    return int(_lib().niorca_batch_workspace_bytes(int(num_graphs), int(total_n), int(total_m)))


def version() -> int:
    return int(_lib().niorca_version())


def profile_enable(on: bool = True) -> None:
    """Per-kernel CUDA-event timing on the launching stream (see niorca.h)."""
    _lib().niorca_profile_enable(1 if on else 0)


def profile_reset() -> None:
    _lib().niorca_profile_reset()


def profile_read() -> dict:
    """{kernel name: (total ms, launches)} accumulated since the last reset."""
    import numpy as np
    k = 64
    ms = np.zeros(k, dtype=np.float64)
    cnt = np.zeros(k, dtype=np.int64)
    nk = _lib().niorca_profile_read(ms.ctypes.data, cnt.ctypes.data, k)
    return {_lib().niorca_kernel_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(nk)}


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(_lib().niorca_launch_count())


TUNING_KEYS = ("grid_relabel", "grid_tri", "grid_agg", "grid_c4", "grid_solve", "long_row_class", "c4_warp_maxw",
               "warp_maxd", "tri_bits_maxd", "tri_hash_maxd", "c4_team_minw")


def get_tuning() -> dict:
    import numpy as np
    v = np.zeros(len(TUNING_KEYS), dtype=np.int32)
    _lib().niorca_get_tuning(v.ctypes.data, len(v))
    return dict(zip(TUNING_KEYS, (int(x) for x in v)))


def set_tuning(**kw) -> None:
    """Set launch-shape knobs by name (see niorca_set_tuning); others keep their value."""
    import numpy as np
    cur = get_tuning()
    for k, val in kw.items():
        if k not in cur:
            raise KeyError(k)
        cur[k] = int(val)
    v = np.array([cur[k] for k in TUNING_KEYS], dtype=np.int32)
    st = _lib().niorca_set_tuning(v.ctypes.data, len(v))
    if st:
        raise NiorcaError(st, "niorca_set_tuning")

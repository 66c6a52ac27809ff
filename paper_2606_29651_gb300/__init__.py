"""GB300-native NI-ORCA: exact per-vertex counts of the 15 non-induced
graphlet orbits on up to four vertices (arxiv 2606.29651), computed by
hand-written sm_103a CUDA kernels behind the C ABI of include/niorca.h.

    import paper_2606_29651_gb300 as ni
    psi = ni.count(rowptr_cuda_int32, colidx_cuda_int32)   # int64 [n, 15]
"""
from ._lib import (NiorcaError, Status, batch_workspace_bytes, check, count, count_batch, count_host,  # noqa: F401
                   count_induced, last_status,
                   get_tuning, launch_count, library, profile_enable, profile_read, profile_reset, set_tuning,
                   validate, version, workspace_bytes)
from .builder import build  # noqa: F401

"""niorca_count_noalloc: counting for callers that cannot allocate device
memory (a host application or framework owns the memory; allocation after
start-up is forbidden). Called through the C ABI with ctypes; its output must
equal niorca_count's (integers: bit-exact) on two calls in a row.

This file is collected last on purpose: it passes alone in a fresh process
and after every other test."""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_29651_gb300 import builder
    h = ctypes.CDLL(builder.build())
    vp = ctypes.c_void_p
    h.niorca_count_noalloc.restype = ctypes.c_int
    h.niorca_count_noalloc.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int64, vp, vp, vp]
    h.niorca_count.restype = ctypes.c_int
    h.niorca_count.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_int64, vp, vp]
    return h


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda:0", dtype=dtype)


def _run(lib, fn, rp, ci, status=None):
    n, m = len(rp) - 1, len(ci)
    r, c = _dev(rp, torch.int32), _dev(ci, torch.int32)
    out = torch.full((n, 15), -1, dtype=torch.int64, device="cuda:0")
    st = torch.cuda.current_stream().cuda_stream
    if fn == "noalloc":
        rc = lib.niorca_count_noalloc(r.data_ptr(), c.data_ptr() if m else None, n, m, out.data_ptr(),
                                      status.data_ptr() if status is not None else None, st)
    else:
        rc = lib.niorca_count(r.data_ptr(), c.data_ptr() if m else None, n, m, out.data_ptr(), st)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name,make", [
    ("er2000", lambda: gg.er(2000, 0.01, 1)),
    ("rmat12", lambda: gg.rmat(12, 16, seed=3)),
    ("k2_12000", lambda: gg.complete_bipartite(2, 12000)),   # the 512-thread 4-cycle tier
    ("k3_9000", lambda: gg.complete_bipartite(3, 9000)),     # the cluster (dense row) 4-cycle tier
])
def test_noalloc_matches_count_on_two_calls(lib, name, make):
    rp, ci = make()
    ref = _run(lib, "count", rp, ci)
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda:0")
    for _ in range(2):
        got = _run(lib, "noalloc", rp, ci, status)
        assert np.array_equal(got, ref), name
        assert int(status.item()) == 0


def test_noalloc_without_status_and_after_another_graph(lib):
    a = gg.er(1500, 0.02, 5)
    b = gg.rmat(10, 16, seed=6)
    ra, rb = _run(lib, "count", *a), _run(lib, "count", *b)
    assert np.array_equal(_run(lib, "noalloc", *a), ra)
    assert np.array_equal(_run(lib, "noalloc", *b), rb)
    assert np.array_equal(_run(lib, "noalloc", *a), ra)


def _scratch_bytes():
    """NIORCA_NOALLOC_SCRATCH_BYTES as include/niorca.h defines it."""
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "niorca.h")
    mt = re.search(r"#define NIORCA_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", open(hdr).read())
    assert mt, "NIORCA_NOALLOC_SCRATCH_BYTES not found in niorca.h"
    return int(mt.group(1)) << int(mt.group(2))


def test_noalloc_rejects_a_graph_beyond_the_static_array(lib):
    # The sizes claim a graph whose column array alone (4 m bytes, twice over
    # in the work memory) is larger than the static array, so the call must
    # refuse it on the host before anything is enqueued; the 8-element
    # buffers are never read. Should the array ever grow past what such a
    # graph needs, the test skips rather than pass undersized buffers.
    scratch = _scratch_bytes()
    n, m = 1_000_000, min(scratch // 2, 2**31 - 2)
    lib.niorca_workspace_bytes.restype = ctypes.c_size_t
    lib.niorca_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64]
    need = lib.niorca_workspace_bytes(n, m)
    if 8 * m <= 2 * scratch or need <= 2 * scratch:
        pytest.skip("the static array is too large for this refusal check")
    small = torch.zeros(8, dtype=torch.int32, device="cuda:0")
    out = torch.zeros(8, dtype=torch.int64, device="cuda:0")
    rc = lib.niorca_count_noalloc(small.data_ptr(), small.data_ptr(), n, m, out.data_ptr(), None,
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 4   # NIORCA_ENOMEM

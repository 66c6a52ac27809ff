"""The C-ABI library builds here and exports every entry point that
include/niorca.h declares (no GPU needed: nothing is called that computes)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "niorca.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(niorca_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_29651_gb300 import builder
    path = builder.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("niorca_count", "niorca_count_batch", "niorca_last_status", "niorca_workspace_bytes"):
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_host_only_entry_points(lib):
    lib.niorca_status_string.restype = ctypes.c_char_p
    lib.niorca_status_string.argtypes = [ctypes.c_int]
    assert lib.niorca_status_string(0) == b"ok"
    assert b"simple" in lib.niorca_status_string(2)
    assert lib.niorca_version() >= 100


def test_argument_errors_are_synchronous(lib):
    # rejected before any CUDA call: negative sizes, null pointers
    lib.niorca_count.restype = ctypes.c_int
    lib.niorca_count.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                 ctypes.c_void_p, ctypes.c_void_p]
    assert lib.niorca_count(None, None, -1, 0, None, None) == 1
    assert lib.niorca_count(None, None, 5, 10, None, None) == 1
    assert lib.niorca_count(None, None, 0, 0, None, None) == 0
    assert lib.niorca_count(None, None, 0, 4, None, None) == 1
    assert lib.niorca_count(None, None, 3, 2**31, None, None) == 1


def test_oracle_and_library_share_no_code():
    csrc = os.path.join(ROOT, "paper_2606_29651_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower().replace("oracle-free", ""), f
    for f in ("_lib.py", "__init__.py", "builder.py"):
        text = open(os.path.join(ROOT, "paper_2606_29651_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text, f

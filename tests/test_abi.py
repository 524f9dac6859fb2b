"""The C ABI library builds for sm_103a, loads and exports every declared call (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lowrank.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:lr_status|const char\*)\s+(lr_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import ctypes

    from paper_1804_07531_gb300 import _binding, build
    if not os.path.exists(_binding.LIB_PATH):
        build.build()
    return ctypes.CDLL(_binding.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lr_sketch", "lr_orth", "lr_subspace_iter", "lr_single_pass", "lr_block_krylov"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1804_07531_gb300 import _binding
    names = _declared()
    assert set(names) == set(_binding.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib):
    import ctypes
    lib.lr_status_string.restype = ctypes.c_char_p
    assert lib.lr_status_string(0) == b"ok"
    assert b"Cholesky" in lib.lr_status_string(5)


def test_null_handle_is_rejected(lib):
    assert lib.lr_sketch(None, None, None, None, None, None, None, None) == 1

"""The C-ABI library builds, loads and exports every entry point that
include/lcs.h declares (no compute calls: this runs without a GPU)."""
import ctypes

import pytest

from paper_2309_09072_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = binding.declared_symbols()
    for required in ["lcs_create", "lcs_destroy", "lcs_strerror", "lcs_length", "lcs_dist",
                     "lcs_strip_dist", "lcs_merge", "lcs_traceback", "lcs_solve", "lcs_solve_host",
                     "lcs_sync", "lcs_get_stats", "lcs_set_strip_height", "lcs_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in binding.declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_strerror_without_gpu(lib):
    lib.lcs_strerror.restype = ctypes.c_char_p
    assert lib.lcs_strerror(0) == b"ok"
    assert b"invalid" in lib.lcs_strerror(1)
    assert lib.lcs_strerror(99) == b"unknown status"


def test_null_arguments_are_rejected(lib):
    # EINVAL before any CUDA call.
    assert lib.lcs_create(None, 0, 0) == 1
    assert lib.lcs_destroy(None) == 1
    assert lib.lcs_get_stats(None, None) == 1
    assert lib.lcs_set_strip_height(None, 4) == 1

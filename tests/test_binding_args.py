"""Argument checks of the Python binding (host logic, no GPU).

The binding hands raw pointers and element counts to the C ABI, so a tensor
of the wrong type, layout or placement would be read as the wrong bytes.
These checks run before any library call, so they are testable on the CPU.
"""
import pytest
import torch

from paper_2309_09072_gb300 import binding as B


def _u8(n):
    return torch.arange(n, dtype=torch.int64).remainder(4).to(torch.uint8)


def test_strings_must_be_contiguous_uint8():
    a = _u8(16)
    with pytest.raises(ValueError, match="contiguous uint8"):
        B._seq(a[::2], "a")
    with pytest.raises(ValueError, match="contiguous uint8"):
        B._seq(a.to(torch.int64), "a")
    ptr, n = B._seq(a, "a", device=False)
    assert n == 16 and ptr.value == a.data_ptr()


def test_device_entry_points_reject_host_tensors():
    a, b = _u8(8), _u8(9)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        B.lcs_solve(None, a, b)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        B.lcs_length(None, a, b)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        B.lcs_path(None, a, b, torch.zeros((4, 2), dtype=torch.int32))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        B.lcs_batch_submit(None, [(a, b)])


def test_output_buffers_checked():
    with pytest.raises(ValueError, match="contiguous int32"):
        B._out(torch.zeros(4, dtype=torch.int64), "cross", torch.int32, device=False)
    with pytest.raises(ValueError, match="contiguous uint8"):
        B._out(torch.zeros((4, 4), dtype=torch.uint8)[:, 1], "out_lcs", torch.uint8, device=False)
    assert B._out(None, "cross", torch.int32) is None


def test_matrices_checked():
    with pytest.raises(ValueError, match="2-D"):
        B._mat(torch.zeros(9, dtype=torch.int32), "dist", device=False)
    with pytest.raises(ValueError, match="unit column stride"):
        B._mat(torch.zeros((5, 8), dtype=torch.int32)[:, ::2], "dist", device=False)
    with pytest.raises(ValueError, match="int32 or int16"):
        B._mat(torch.zeros((5, 8), dtype=torch.float32), "dist", device=False)
    assert B._mat(torch.zeros((5, 8), dtype=torch.int16), "dist", device=False) == 8
    # A padded leading dimension is legal: ld is the row stride.
    assert B._mat(torch.zeros((5, 12), dtype=torch.int32)[:, :5], "dist", device=False) == 12


def test_host_entry_point_takes_host_tensors():
    # lcs_solve_host's strings and outputs must live on the host; a host
    # tensor passes the check (the call itself needs the library and a GPU).
    ptr, n = B._seq(_u8(5), "a_host", device=False)
    assert n == 5
    with pytest.raises(ValueError, match="host"):
        B._place(type("FakeCuda", (), {"is_cuda": True})(), "a_host", device=False)

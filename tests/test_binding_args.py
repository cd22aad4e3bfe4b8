"""Argument checks of the Python binding (host logic only, no GPU): the tensors handed to the C ABI
as raw pointers must be contiguous float32 of the expected shape, on the device the call expects
(host memory for gs_iterate_host's target and loss)."""
import pytest
import torch

from paper_2504_02437_gb300 import api


def test_host_tensor_accepted_and_rejected():
    t = torch.zeros(2, 3, 4, 5)
    assert api._f32(t, (2, 3, 4, 5), "target", host=True) is t
    assert api._hptr(t).value == t.data_ptr()
    assert api._f32(None, (3,), "loss_out", host=True) is None and api._hptr(None) is None
    with pytest.raises(ValueError, match="expected float32"):
        api._f32(t.double(), (2, 3, 4, 5), "target", host=True)
    with pytest.raises(ValueError, match="expected float32"):
        api._f32(t, (2, 3, 4, 6), "target", host=True)
    strided = torch.zeros(2, 3, 5, 4).transpose(2, 3)
    with pytest.raises(ValueError, match="contiguous"):
        api._f32(strided, (2, 3, 4, 5), "target", host=True)
    with pytest.raises(ValueError, match="contiguous host"):
        api._hptr(strided)


def test_device_tensor_expected_where_the_call_reads_device_memory():
    t = torch.zeros(3)
    with pytest.raises(ValueError, match="CUDA tensor"):
        api._f32(t, (3,), "loss_out")
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        api._ptr(t)

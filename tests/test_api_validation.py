"""Argument checks of the Python layer that run before the library is called
(no GPU): an `out` buffer of the wrong shape, element type or device, or a
non-contiguous tensor, for the entry points that hand plain pointers and one
element type to the library, must raise instead of reaching a kernel."""
import pytest
import torch

from paper_1002_2184_gb300 import api


def test_filter_rejects_mismatched_out():
    x = torch.zeros(4, 64, dtype=torch.float64)
    with pytest.raises(ValueError, match="dtype"):
        api.filter_dwt1d(x, 2, out=torch.zeros(4, 64, dtype=torch.float32))
    with pytest.raises(ValueError, match="shape"):
        api.filter_dwt1d(x, 2, out=torch.zeros(4, 32, dtype=torch.float64))
    with pytest.raises(ValueError, match="dtype"):
        api.filter_idwt1d(x, 2, out=torch.zeros(4, 64, dtype=torch.float32))


def test_filter_rejects_non_contiguous_and_host_tensors():
    x = torch.zeros(64, 4).t()
    with pytest.raises(ValueError, match="contiguous"):
        api.filter_dwt1d(x, 2)
    with pytest.raises(ValueError, match="CUDA"):
        api.filter_dwt1d(torch.zeros(4, 64), 2)


def test_undecimated_rejects_mismatched_out():
    x = torch.zeros(3, 128)
    with pytest.raises(ValueError, match="shape"):
        api.swt1d(x, 2, out=torch.zeros(3, 2, 128))  # needs levels + 1 = 3 bands
    with pytest.raises(ValueError, match="dtype"):
        api.swt1d(x, 2, out=torch.zeros(3, 3, 128, dtype=torch.float64))
    c = torch.zeros(3, 3, 128)
    with pytest.raises(ValueError, match="bands|expected"):
        api.iswt1d(c, 4)  # 3 bands is not levels + 1 = 5
    with pytest.raises(ValueError, match="shape"):
        api.iswt1d(c, 2, out=torch.zeros(3, 64))
    with pytest.raises(ValueError, match="CUDA"):
        api.iswt1d(c, 2)


def test_out_on_another_device_is_rejected():
    x = torch.zeros(2, 64, 64)
    with pytest.raises(ValueError, match="meta"):
        api.dwt2d(x, 2, out=torch.empty(2, 64, 64, device="meta"))
    with pytest.raises(ValueError, match="meta"):
        api.filter_dwt1d(torch.zeros(2, 64), 2, out=torch.empty(2, 64, device="meta"))


def test_plan_rejects_buffers_on_another_device():
    x = torch.zeros(2, 64, 64)
    with pytest.raises(ValueError, match="meta"):
        api.Plan(x, torch.empty(2, 64, 64, device="meta"), 2)

"""Argument checks of the Python binding that run before any context or
launch: result buffers of the wrong dtype, shape or device, and device tensors
given to the host-buffer call, are refused instead of being read as raw memory."""
import numpy as np
import pytest
import torch

from paper_2609_03866_b300 import api

OFFS = np.array([0, 4, 9], dtype=np.int64)
T = np.array([0.0, 1.0, 2.5, 4.0, 0.0, 0.5, 1.0, 3.0, 7.0])
X = np.array([1.0, -2.0, 0.5, 3.0, 2.0, 1.0, -1.0, 0.0, 4.0])
LAGS = np.array([0.0, 1.0, 2.0])


def host_out(**over):
    out = {"c": torch.empty(2, 3, dtype=torch.float64), "b": torch.empty(2, 3, dtype=torch.float64),
           "count": torch.empty(2, 3, dtype=torch.int64)}
    out.update(over)
    return out


@pytest.mark.parametrize("key,bad", [
    ("c", torch.empty(2, 3, dtype=torch.float32)),      # wrong dtype
    ("c", torch.empty(3, 2, dtype=torch.float64)),      # wrong shape
    ("b", torch.empty(2, 3, dtype=torch.float64).t().contiguous().t()),  # not contiguous
    ("count", torch.empty(2, 3, dtype=torch.int32)),    # counts are int64
    ("c", None),                                        # c is required
])
def test_host_call_refuses_bad_result_buffers(key, bad):
    with pytest.raises(ValueError):
        api.corr_batch_host(OFFS, T, X, LAGS, kernel="rectangle", h=0.5, out=host_out(**{key: bad}))


def test_check_out_accepts_optional_buffers_left_out():
    api._check_out({"c": torch.empty(2, 3, dtype=torch.float64)}, (2, 3), "cpu")
    api._check_out(host_out(), (2, 3), "cpu")


def test_check_device_input_wants_float64_of_the_planned_size():
    good = torch.zeros(9, dtype=torch.float64)
    api._check_device_input("t", good, 9, "cpu")
    for bad in (torch.zeros(9, dtype=torch.float32), torch.zeros(8, dtype=torch.float64),
                torch.zeros(18, dtype=torch.float64)[::2], np.zeros(9)):
        with pytest.raises(ValueError):
            api._check_device_input("t", bad, 9, "cpu")


def test_multi_host_call_refuses_mismatched_result_buffers():
    opts = [dict(kernel="rectangle", h=0.5), dict(kernel="gaussian", h=0.5)]
    with pytest.raises(ValueError):   # one dict of buffers per option set
        api.corr_batch_host_multi(OFFS, T, X, LAGS, opts, outs=[host_out()])
    with pytest.raises(ValueError):
        api.corr_batch_host_multi(OFFS, T, X, LAGS, opts, outs=[host_out(), host_out(c=torch.empty(2, 2))])
    with pytest.raises(ValueError):
        api.corr_batch_host_multi(OFFS, T, X, LAGS, [])

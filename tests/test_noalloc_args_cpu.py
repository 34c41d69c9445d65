"""Argument checks of the allocation-free block inverse's binding (CPU).

Every operand that would make a kernel read or write the wrong memory must
be refused before a pointer reaches the library: host arrays, tensors of the
wrong dtype or of two different devices or dtypes, buffers smaller than
s * s, and an s that cannot be inferred.  A stand-in object with the
attributes of a CUDA tensor lets these run without a GPU; nothing here calls
the library.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_1708_04539_gb300.binding import NOALLOC_MAX_S, _noalloc_args, F64, C128


class FakeCudaTensor:
    def __init__(self, shape, dtype=torch.float64, device="cuda:0", contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = torch.device(device)
        self.is_cuda = True
        self._contig = contiguous

    def dim(self):
        return len(self.shape)

    def numel(self):
        return int(np.prod(self.shape)) if self.shape else 1

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        raise AssertionError("a refused operand must never have its pointer taken")


def test_accepts_square_and_flat_buffers():
    assert _noalloc_args(FakeCudaTensor((12, 12)), FakeCudaTensor((12, 12)), None) == (12, F64)
    assert _noalloc_args(FakeCudaTensor((144,), torch.complex128),
                         FakeCudaTensor((144,), torch.complex128), None) == (12, C128)
    assert _noalloc_args(FakeCudaTensor((200,)), FakeCudaTensor((100,)), 10) == (10, F64)


def test_refuses_host_arrays():
    with pytest.raises(TypeError):
        _noalloc_args(np.eye(4), FakeCudaTensor((4, 4)), None)
    with pytest.raises(TypeError):
        _noalloc_args(FakeCudaTensor((4, 4)), np.eye(4), None)


def test_refuses_cpu_tensors():
    with pytest.raises(ValueError):
        _noalloc_args(torch.eye(4, dtype=torch.float64), FakeCudaTensor((4, 4)), None)


@pytest.mark.parametrize("dtype", [torch.float32, torch.complex64, torch.int64])
def test_refuses_other_dtypes(dtype):
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 4), dtype), FakeCudaTensor((4, 4), dtype), None)


def test_refuses_mixed_dtypes_and_devices():
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 4)), FakeCudaTensor((4, 4), torch.complex128), None)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 4)), FakeCudaTensor((4, 4), device="cuda:1"), None)


def test_refuses_short_buffers_and_bad_sizes():
    # the flat layout get_selected returns: s must not be read off shape[0]
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((99,)), FakeCudaTensor((99,)), None)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((100,)), FakeCudaTensor((100,)), 11)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 5)), FakeCudaTensor((4, 5)), None)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((300, 300)), FakeCudaTensor((300, 300)), NOALLOC_MAX_S + 1)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 4)), FakeCudaTensor((4, 4)), 0)
    with pytest.raises(ValueError):
        _noalloc_args(FakeCudaTensor((4, 4), contiguous=False), FakeCudaTensor((4, 4)), None)

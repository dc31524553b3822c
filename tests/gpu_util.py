"""Helpers for the GPU tests: device buffers through torch, conversions, relative errors."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def to_dev(a):
    """complex numpy array -> torch float tensor (interleaved re/im) on cuda:0."""
    torch = torch_cuda()
    a = np.ascontiguousarray(a)
    if a.dtype == np.complex128:
        return torch.from_numpy(a.view(np.float64).copy()).cuda()
    if a.dtype == np.complex64:
        return torch.from_numpy(a.view(np.float32).copy()).cuda()
    return torch.from_numpy(a.copy()).cuda()


def from_dev(t, shape, dtype=np.complex128):
    torch = torch_cuda()
    torch.cuda.synchronize()
    h = t.cpu().numpy()
    return h.view(dtype).reshape(shape)


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())

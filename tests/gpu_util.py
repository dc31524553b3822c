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


def coarse_from_bundle(arr, nsys, nc, Vc):
    """FP32 coarse bundle [ntile][nc][Vc][2][2] (flat numpy float32) -> complex128 [nsys][Vc][nc]."""
    nt = (nsys + 1) // 2
    a = arr.reshape(nt, nc, Vc, 2, 2)
    out = np.empty((nsys, Vc, nc), dtype=np.complex128)
    for n in range(nsys):
        t, l = divmod(n, 2)
        out[n] = (a[t, :, :, 0, l] + 1j * a[t, :, :, 1, l]).T
    return out


def coarse_to_bundle(x, nc, Vc):
    """complex [nsys][Vc][nc] -> FP32 coarse bundle (flat numpy float32)."""
    nsys = x.shape[0]
    nt = (nsys + 1) // 2
    a = np.zeros((nt, nc, Vc, 2, 2), dtype=np.float32)
    for n in range(nsys):
        t, l = divmod(n, 2)
        a[t, :, :, 0, l] = x[n].T.real
        a[t, :, :, 1, l] = x[n].T.imag
    return a.ravel()


class Lattice:
    """A context with a gauge field and operator on cuda:0, plus helpers for fine bundles."""

    def __init__(self, L, U, kappa, c_sw, bc_t=-1):
        self.torch = torch_cuda()
        from paper_2201_03872_gb300 import tmamg as T
        self.T = T
        self.L = L
        self.V = int(np.prod(L))
        self.ctx = T.tmamg_create(L, bc_t)
        T.tmamg_load_gauge(self.ctx, U)
        T.tmamg_set_operator(self.ctx, kappa, c_sw)

    def close(self):
        self.T.tmamg_destroy(self.ctx)

    def fine_bundle(self, x):
        """complex [nsys, ...fine] -> FP32 bundle tensor"""
        torch = self.torch
        nsys = x.shape[0]
        xf = to_dev(np.ascontiguousarray(x.astype(np.complex64)))
        nb = self.T.tmamg_bundle_bytes(self.ctx, nsys, 32)
        b = torch.zeros(nb // 4, dtype=torch.float32, device="cuda")
        self.T.tmamg_pack(self.ctx, xf, b, nsys, 32)
        return b

    def from_fine_bundle(self, b, nsys):
        torch = self.torch
        L = self.L
        f = torch.empty(nsys * self.V * 24, dtype=torch.float32, device="cuda")
        self.T.tmamg_unpack(self.ctx, b, f, nsys, 32)
        return from_dev(f, (nsys, L[3], L[2], L[1], L[0], 4, 3), np.complex64).astype(np.complex128)

    def coarse_buffer(self, nsys, level=1):
        nb = self.T.tmamg_coarse_bundle_bytes(self.ctx, level, nsys)
        return self.torch.zeros(nb // 4, dtype=torch_cuda().float32, device="cuda")

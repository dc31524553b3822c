"""GPU coarse-level solvers (persistent GMRES, block GMRES per shift, per-launch GMRES)
against the FP64 oracle on the same Galerkin coarse operator (test vectors injected).

* k-step iterates: with the stopping test disabled, k steps of each GPU solver equal k
  steps of the oracle's GMRES (or block GMRES over the right-hand sides of one shift) up to
  FP32 rounding through k Arnoldi steps (bar 1e-4 relative).
* converged solves reach the requested coarse residual, checked with the oracle operator.
* the block solver needs no more steps than the per-system solver (paper Sec. 4: block
  Krylov reduces the bottom-level iteration count)."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac, krylov
from tests.gpu_util import Lattice, coarse_from_bundle, coarse_to_bundle, relerr, to_dev

pytestmark = pytest.mark.gpu

L = (8, 4, 4, 8)
AGG = (4, 2, 2, 4)
NV = 8


@pytest.fixture(scope="module")
def coarse():
    U = synth.gauge_field(L, 0.3, seed=101)
    kappa = 0.125
    lat = Lattice(L, U, kappa, 1.0)
    Vt = synth.gaussian_spinors(L, NV, seed=102).astype(np.complex64)
    p = lat.T.setup_params(agg=AGG, nv=NV, sap_block=(2, 2, 2, 2), setup_iters=0)
    lat.T.tmamg_setup_from_vectors(lat.ctx, p, to_dev(Vt))
    op = dirac.Operator(U, kappa, 1.0)
    P = amg.Prolongation(amg.FineLevel.to_chi(Vt.astype(np.complex128)), L, AGG)
    cl = amg.CoarseLevel(amg.coarse_operator(amg.FineLevel(op), P), P.Lc, NV)
    yield lat, cl, P
    lat.close()


def _run(lat, cl, rc, nrhs, mus, solver, tol, restart, maxiter):
    T = lat.T
    nc, Vc = 2 * NV, int(np.prod(cl.L))
    nsys = nrhs * len(mus)
    rb = lat.torch.from_numpy(coarse_to_bundle(rc, nc, Vc)).cuda()
    xb = lat.torch.zeros_like(rb)
    sp = T.solve_params(coarse_solver=solver, coarse_tol=tol, coarse_restart=restart, coarse_maxiter=maxiter)
    it = T.tmamg_coarse_solve(lat.ctx, 1, rb, xb, nrhs, mus, len(mus), sp)
    lat.torch.cuda.synchronize()
    return coarse_from_bundle(xb.cpu().numpy(), nsys, nc, Vc), it


def _shape(cl, v):
    Lxc, Lyc, Lzc, Ltc = cl.L
    return v.reshape(Ltc, Lzc, Lyc, Lxc, 2, NV)


@pytest.mark.parametrize("solver", [0, 2])
def test_gmres_k_steps_match_oracle(coarse, solver):
    lat, cl, P = coarse
    nrhs, mus = 3, [0.01, 0.2]
    nsys = nrhs * len(mus)
    Vc, nc = int(np.prod(cl.L)), 2 * NV
    rc = synth.complex_normal(103, 1, (nsys, Vc, nc))
    k = 8
    x, it = _run(lat, cl, rc, nrhs, mus, solver, 1e-30, 16, k)
    assert it == k
    for n in range(nsys):
        mu = mus[n % len(mus)]
        A = lambda v: cl.apply(_shape(cl, v), mu).ravel()
        xr, _ = krylov.fgmres(A, rc[n].ravel(), tol=1e-30, restart=16, maxiter=k)
        assert relerr(x[n].ravel(), xr) < 1e-4, (n, relerr(x[n].ravel(), xr))


def test_block_gmres_k_steps_match_oracle(coarse):
    lat, cl, P = coarse
    nrhs, mus = 3, [0.01, 0.2]
    nsys = nrhs * len(mus)
    Vc, nc = int(np.prod(cl.L)), 2 * NV
    rc = synth.complex_normal(104, 1, (nsys, Vc, nc))
    k = 5
    x, it = _run(lat, cl, rc, nrhs, mus, 1, 1e-30, 16, k)
    assert it == k
    for kk, mu in enumerate(mus):
        idx = [r * len(mus) + kk for r in range(nrhs)]
        A = lambda v: cl.apply(_shape(cl, v), mu).ravel()
        B = np.stack([rc[n].ravel() for n in idx], axis=1)
        X, _ = krylov.block_gmres(A, B, tol=1e-30, restart=16, maxiter=k)
        for c, n in enumerate(idx):
            assert relerr(x[n].ravel(), X[:, c]) < 1e-4, (n, relerr(x[n].ravel(), X[:, c]))


@pytest.mark.parametrize("solver", [0, 1, 2])
def test_converged_coarse_solve(coarse, solver):
    lat, cl, P = coarse
    nrhs, mus = 4, [0.001, 0.05]
    nsys = nrhs * len(mus)
    Vc, nc = int(np.prod(cl.L)), 2 * NV
    rc = synth.complex_normal(105, 1, (nsys, Vc, nc))
    x, it = _run(lat, cl, rc, nrhs, mus, solver, 1e-5, 20, 400)
    for n in range(nsys):
        mu = mus[n % len(mus)]
        res = np.linalg.norm(rc[n].ravel() - cl.apply(_shape(cl, x[n]), mu).ravel()) / np.linalg.norm(rc[n])
        assert res < 2e-5, (solver, n, res)


def test_block_needs_no_more_steps(coarse):
    lat, cl, P = coarse
    nrhs, mus = 6, [0.001]
    Vc, nc = int(np.prod(cl.L)), 2 * NV
    rc = synth.complex_normal(106, 1, (nrhs, Vc, nc))
    _, it_block = _run(lat, cl, rc, nrhs, mus, 1, 1e-1, 40, 400)
    _, it_gmres = _run(lat, cl, rc, nrhs, mus, 0, 1e-1, 40, 400)
    assert it_block <= it_gmres, (it_block, it_gmres)

"""GPU parity of the non-degenerate twisted-mass doublet (operator and multigrid solve) against the
FP64 oracle.

The doublet D_ND(mu, eps) = D_W (x) 1 + i mu gamma5 (x) tau3 - eps 1 (x) tau1 acts on a pair (u, d)
as (D(mu) u - eps d, D(-mu) d - eps u). Bars: the stencil's own (relative 1e-13 in FP64, 1e-6 in
FP32, per doublet); the solver's FP64 true residual at its tolerance, checked through the oracle."""
import numpy as np
import pytest

import synth
from oracle import dirac, doublet
from tests.gpu_util import Lattice, torch_cuda, to_dev, from_dev, relerr

pytestmark = pytest.mark.gpu

TOL = {64: 1e-13, 32: 1e-6}


def _site_shape(L):
    return (L[3], L[2], L[1], L[0], 4, 3)


def _doublet_apply(lat, u, d, mu, eps, prec):
    """GPU D_ND on fields u, d [npair, ...]: packs [npair][2] fields into a bundle of 2 npair systems."""
    torch = lat.torch
    T = lat.T
    npair = u.shape[0]
    nsys = 2 * npair
    cdt = np.complex128 if prec == 64 else np.complex64
    f = np.stack([u, d], axis=1).reshape((nsys,) + u.shape[1:]).astype(cdt)
    xf = to_dev(f)
    rdt = torch.float64 if prec == 64 else torch.float32
    nb = T.tmamg_bundle_bytes(lat.ctx, nsys, prec) // (8 if prec == 64 else 4)
    xb = torch.zeros(nb, dtype=rdt, device="cuda")
    yb = torch.zeros(nb, dtype=rdt, device="cuda")
    T.tmamg_pack(lat.ctx, xf, xb, nsys, prec)
    T.tmamg_dirac_doublet(lat.ctx, xb, yb, npair, mu, eps, prec)
    yf = torch.zeros_like(xf)
    T.tmamg_unpack(lat.ctx, yb, yf, nsys, prec)
    y = from_dev(yf, f.shape, cdt).astype(np.complex128).reshape((npair, 2) + u.shape[1:])
    return y[:, 0], y[:, 1], (xb, yb)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("bc_t", [-1, 1])
def test_doublet_operator_matches_oracle(prec, bc_t):
    L = (8, 4, 4, 6)
    U = synth.gauge_field(L, 0.3, seed=91)
    kappa, c_sw = 0.127, 1.0
    lat = Lattice(L, U, kappa, c_sw, bc_t)
    try:
        npair = 3
        x = synth.gaussian_spinors(L, 2 * npair, seed=92)
        u, d = x[0::2], x[1::2]
        mu = np.array([0.003, -0.05, 0.2])
        eps = np.array([0.15, 0.0, 0.4])
        yu, yd, _ = _doublet_apply(lat, u, d, mu, eps, prec)
        op = dirac.Operator(U, kappa, c_sw, bc_t)
        for q in range(npair):
            ru, rd = doublet.apply(op, u[q], d[q], mu[q], eps[q])
            err = np.sqrt(np.linalg.norm(yu[q] - ru) ** 2 + np.linalg.norm(yd[q] - rd) ** 2)
            ref = np.sqrt(np.linalg.norm(ru) ** 2 + np.linalg.norm(rd) ** 2)
            assert err / ref <= TOL[prec], (q, err / ref)
    finally:
        lat.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_doublet_without_splitting_is_two_degenerate_systems(prec):
    # eps = 0: the flavours decouple into D(mu) u and D(-mu) d, the degenerate stencil bit for bit
    torch = torch_cuda()
    L = (4, 4, 4, 8)
    U = synth.gauge_field(L, 0.3, seed=93)
    lat = Lattice(L, U, 0.125, 1.0)
    T = lat.T
    try:
        npair = 2
        x = synth.gaussian_spinors(L, 2 * npair, seed=94)
        mu = np.array([0.01, 0.3])
        _, _, (xb, yb) = _doublet_apply(lat, x[0::2], x[1::2], mu, np.zeros(npair), prec)
        y2 = torch.zeros_like(yb)
        T.tmamg_dirac(lat.ctx, xb, y2, 2 * npair, np.array([mu[0], -mu[0], mu[1], -mu[1]]), prec)
        torch.cuda.synchronize()
        assert torch.equal(yb, y2)
    finally:
        lat.close()


def _solve_doublet(L, U, kappa, b, mus, epss, sp_kw, solve_kw):
    lat = Lattice(L, U, kappa, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(**sp_kw))
        nrhs = b.shape[0]
        x = np.zeros((nrhs, len(mus)) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve_doublet(lat.ctx, b, nrhs, mus, epss, len(mus), x, 0, T.solve_params(**solve_kw))
        return rc, stats, x
    finally:
        lat.close()


def _check_doublet_residuals(op, b, x, mus, epss, stats, tol):
    for r in range(b.shape[0]):
        bn = np.sqrt(np.linalg.norm(b[r, 0]) ** 2 + np.linalg.norm(b[r, 1]) ** 2)
        for k, (mu, eps) in enumerate(zip(mus, epss)):
            yu, yd = doublet.apply(op, x[r, k, 0], x[r, k, 1], mu, eps)
            res = np.sqrt(np.linalg.norm(b[r, 0] - yu) ** 2 + np.linalg.norm(b[r, 1] - yd) ** 2) / bn
            s = stats[r * len(mus) + k]
            assert res <= tol, (r, k, res)
            assert s.status == 0 and abs(s.true_rel_res - res) < 0.1 * tol, (r, k, s.true_rel_res, res)


@pytest.mark.parametrize("coarse_precision", [16, 32])
def test_solve_doublet_two_level(coarse_precision):
    L = (8, 4, 4, 8)
    U = synth.gauge_field(L, 0.3, seed=95)
    kappa = 0.126
    nrhs = 2
    b = synth.gaussian_spinors(L, 2 * nrhs, seed=96).reshape((nrhs, 2) + _site_shape(L))
    mus = [0.002, 0.05]
    epss = [0.12, 0.3]
    rc, stats, x = _solve_doublet(L, U, kappa, b, mus, epss,
                                  dict(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4),
                                  dict(restart=10, tol=1e-10, coarse_precision=coarse_precision))
    assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
    assert len(stats) == nrhs * len(mus)
    _check_doublet_residuals(dirac.Operator(U, kappa, 1.0), b, x, mus, epss, stats, 1e-10)


def test_solve_doublet_tiny_matches_dense_inverse():
    # 4 x 4 x 2 x 4 lattice: the doublet as a dense (3072 x 3072) matrix, solved directly
    L = (4, 4, 2, 4)
    U = synth.gauge_field(L, 0.3, seed=97)
    kappa = 0.125
    b = synth.gaussian_spinors(L, 2, seed=98).reshape((1, 2) + _site_shape(L))
    mu, eps = 0.01, 0.2
    rc, stats, x = _solve_doublet(L, U, kappa, b, [mu], [eps],
                                  dict(agg=(2, 2, 1, 2), nv=6, sap_block=(2, 2, 1, 2), setup_iters=3),
                                  dict(restart=10, tol=1e-11))
    op = dirac.Operator(U, kappa, 1.0)
    assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
    M = doublet.dense(op, mu, eps)
    xd = np.linalg.solve(M, np.concatenate([b[0, 0].ravel(), b[0, 1].ravel()]))
    got = np.concatenate([x[0, 0, 0].ravel(), x[0, 0, 1].ravel()])
    assert np.linalg.norm(got - xd) <= np.linalg.cond(M) * 1e-11 * np.linalg.norm(xd)


def test_solve_doublet_three_level():
    L = (8, 8, 8, 8)
    U = synth.gauge_field(L, 0.3, seed=99)
    kappa = 0.126
    b = synth.gaussian_spinors(L, 2, seed=100).reshape((1, 2) + _site_shape(L))
    mus = [0.001, 0.04]
    epss = [0.1, 0.2]
    lat = Lattice(L, U, kappa, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(levels=3, agg=(2, 2, 2, 2), nv=8, agg2=(2, 2, 2, 2), nv2=8,
                                              sap_block=(2, 2, 2, 2), setup_iters=4))
        x = np.zeros((1, 2) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve_doublet(lat.ctx, b, 1, mus, epss, 2, x, 0, T.solve_params(restart=10, tol=1e-10))
    finally:
        lat.close()
    assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
    _check_doublet_residuals(dirac.Operator(U, kappa, 1.0), b, x, mus, epss, stats, 1e-10)


def test_solve_doublet_rejects_unsupported_forms():
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, 0.3, seed=101)
    lat = Lattice(L, U, 0.125, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(agg=(2, 2, 2, 2), nv=6, sap_block=(2, 2, 2, 2), setup_iters=1))
        b = np.zeros((1, 2) + _site_shape(L), dtype=np.complex128)
        x = np.zeros_like(b)
        for kw in (dict(precision=64), dict(coarse_solver=1), dict(use_nn=2)):
            with pytest.raises(T.TmamgError):
                T.tmamg_solve_doublet(lat.ctx, b, 1, [0.01], [0.1], 1, x, 0, T.solve_params(**kw))
    finally:
        lat.close()

"""Pins for the oracle multigrid: P, R = P^dagger, D_c = P^dagger D P, two-grid exactness,
and an end-to-end FGMRES-AMG solve on the tiny configuration (4^4, kappa 0.125, c_sw 1,
mu 0.01, 2^4 aggregates, Nv 8, SAP blocks 2^4, FGMRES(10) to 1e-10) against dense inversion."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac
from oracle.gamma import gamma5

L1 = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def tiny():
    U = synth.gauge_field(L1, 0.3, seed=1)
    op = dirac.Operator(U, kappa=0.125, c_sw=1.0, bc_t=-1)
    V0 = synth.gaussian_spinors(L1, 8, seed=1, stream=301)
    mg = amg.TwoLevelAMG(op, agg=(2, 2, 2, 2), V0=V0, sap_block=(2, 2, 2, 2), setup_iters=3)
    Pd = mg.P.dense()
    op.D0 = op.dense(0.0)  # cached dense D(0); D(mu) = D(0) + i mu gamma5 is pinned separately
    return op, mg, Pd


def _dense(op, mu):
    g5 = np.kron(np.eye(op.D0.shape[0] // 12), np.kron(gamma5(), np.eye(3)))
    return op.D0 + 1j * mu * g5


def test_P_orthonormal(tiny):
    op, mg, Pd = tiny
    assert Pd.shape == (3072, 16 * 16)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13


def test_P_preserves_chirality(tiny):
    # P^dagger gamma5 P = gamma5_c = diag(+1 x Nv, -1 x Nv) on every coarse site
    op, mg, Pd = tiny
    g5 = np.kron(np.eye(256), np.kron(gamma5(), np.eye(3)))
    g5c = np.kron(np.eye(16), np.diag([1.0] * 8 + [-1.0] * 8))
    assert np.abs(Pd.conj().T @ g5 @ Pd - g5c).max() < 1e-13


def test_restrict_prolong_are_adjoint(tiny):
    op, mg, Pd = tiny
    r = synth.gaussian_spinors(L1, 1, seed=31)[0]
    rc = mg.P.restrict(amg.FineLevel.to_chi(r))
    assert np.abs(rc.ravel() - Pd.conj().T @ r.ravel()).max() < 1e-13
    e = mg.P.prolong(rc)
    assert np.abs(e.ravel() - Pd @ rc.ravel()).max() < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.01, -0.3])
def test_coarse_operator_is_galerkin(tiny, mu):
    op, mg, Pd = tiny
    Dc = mg.coarse.dense(mu)
    G = Pd.conj().T @ _dense(op, mu) @ Pd
    assert np.abs(Dc - G).max() < 1e-12 * np.abs(G).max()


def test_coarse_twist_is_diagonal(tiny):
    op, mg, Pd = tiny
    d = mg.coarse.dense(0.2) - mg.coarse.dense(0.0)
    g5c = np.kron(np.eye(16), np.diag([1.0] * 8 + [-1.0] * 8))
    assert np.abs(d - 0.2j * g5c).max() < 1e-14


def test_coarse_gamma5_hermiticity(tiny):
    # inherited from the fine operator: gamma5_c D_c(mu) gamma5_c = D_c(-mu)^dagger
    op, mg, Pd = tiny
    g5c = np.kron(np.eye(16), np.diag([1.0] * 8 + [-1.0] * 8))
    mu = 0.05
    assert np.abs(g5c @ mg.coarse.dense(mu) @ g5c - mg.coarse.dense(-mu).conj().T).max() < 1e-13


def test_two_grid_exact_with_unitary_P():
    # single-site aggregates with Nv = 6: P is unitary, so P D_c^{-1} P^dagger = D^{-1}
    # and one cycle with an exact coarse solve returns the exact solution
    Ls = (2, 2, 2, 2)
    op = dirac.Operator(synth.gauge_field(Ls, 0.3, seed=3), kappa=0.125, c_sw=1.0)
    V0 = synth.gaussian_spinors(Ls, 6, seed=3, stream=301)
    mg = amg.TwoLevelAMG(op, agg=(1, 1, 1, 1), V0=V0, sap_block=(1, 1, 1, 2), setup_iters=1)
    r = synth.gaussian_spinors(Ls, 1, seed=32)[0]
    mu = 0.01
    e = mg.cycle(r, mu, coarse_mode="exact")
    x = np.linalg.solve(op.dense(mu), r.ravel())
    assert np.linalg.norm(e.ravel() - x) < 1e-11 * np.linalg.norm(x)


def test_amg_solve_tiny_config(tiny):
    op, mg, Pd = tiny
    b = synth.gaussian_spinors(L1, 1, seed=1, stream=202)[0]
    mu = 0.01
    x, info = mg.solve(b, mu, tol=1e-10, restart=10, maxiter=300)
    assert info["converged"]
    res = np.linalg.norm(b - op.apply(x, mu)) / np.linalg.norm(b)
    assert res <= 1e-10
    M = _dense(op, mu)
    xd = np.linalg.solve(M, b.ravel())
    cond = np.linalg.cond(M)
    assert np.linalg.norm(x.ravel() - xd) <= cond * 1e-10 * np.linalg.norm(xd)
    # the AMG preconditioner must beat unpreconditioned GMRES(10) by a wide margin
    assert info["iters"] < 40

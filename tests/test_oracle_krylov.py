"""Pins for the oracle Krylov solvers against dense linear algebra and exact-arithmetic facts."""
import numpy as np

import synth
from oracle import krylov


def _system(n, seed, shift=4.0):
    # random part has spectral radius ~1; the shift sets the distance of the spectrum from 0
    A = synth.complex_normal(seed, 1, (n, n)) / np.sqrt(n) + shift * np.eye(n)
    b = synth.complex_normal(seed, 2, (n,))
    return A, b


def test_fgmres_matches_dense_solve():
    A, b = _system(60, 1, shift=1.5)
    x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-12, restart=15, maxiter=500)
    assert info["converged"]
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_full_gmres_terminates_in_n_steps():
    # without restarts GMRES reaches the exact solution in at most n steps
    n = 12
    A, b = _system(n, 2, shift=1.2)
    x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-11, restart=n, maxiter=n)
    assert info["iters"] <= n
    assert info["resid"] < 1e-9


def test_fgmres_with_exact_preconditioner_one_step():
    A, b = _system(30, 3)
    Ainv = np.linalg.inv(A)
    x, info = krylov.fgmres(lambda v: A @ v, b, tol=1e-12, restart=5, M=lambda v: Ainv @ v)
    assert info["iters"] == 1 and info["converged"]


def test_block_gmres_s1_equals_gmres():
    A, b = _system(40, 4, shift=1.5)
    for k in (1, 3, 7):
        x1, _ = krylov.fgmres(lambda v: A @ v, b, tol=1e-30, restart=k, maxiter=k)
        X, _ = krylov.block_gmres(lambda v: A @ v, b[:, None], tol=1e-30, restart=k, maxiter=k)
        assert np.linalg.norm(X[:, 0] - x1) < 1e-11 * np.linalg.norm(x1)


def test_block_gmres_dense_block_steps_bound():
    # a block Krylov space of block width s reaches dimension n after ceil(n/s) steps
    n, s = 24, 4
    A, _ = _system(n, 5, shift=1.5)
    B = synth.complex_normal(5, 3, (n, s))
    X, info = krylov.block_gmres(lambda v: A @ v, B, tol=1e-10, restart=n, maxiter=n)
    assert info["iters"] <= int(np.ceil(n / s))
    assert np.linalg.norm(X - np.linalg.solve(A, B)) < 1e-8 * np.linalg.norm(X)


def test_block_gmres_restarted_converges():
    A, _ = _system(80, 6, shift=1.5)
    B = synth.complex_normal(6, 3, (80, 3))
    X, info = krylov.block_gmres(lambda v: A @ v, B, tol=1e-11, restart=6, maxiter=300)
    assert info["converged"]
    R = B - A @ X
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-11 * np.linalg.norm(B, axis=0))

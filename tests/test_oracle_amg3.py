"""Pins for the oracle's second coarse level and three-level cycle: P2 orthonormal and
chirality-preserving, D_c2 = P2^+ D_c1 P2 (dense brute force, on a coarse lattice with extents
3, 2 and 1), the minimal-residual smoother against its one-dimensional least-squares definition,
the coarse inverse iteration against a dense solve, the three-level cycle against the two-level
cycle with an exact coarse solve, and an end-to-end three-level solve against dense inversion."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac


def _random_level(Lc, nv, seed):
    nc = 2 * nv
    A = synth.complex_normal(seed, 401, (9,) + synth.lattice_shape(Lc) + (nc, nc)) * 0.3
    # a dominant self block keeps the level well conditioned (for the iterative pins)
    A[0] += 4.0 * np.eye(nc)
    return amg.CoarseLevel(A, Lc, nv)


def _g5c(nsite, nv):
    return np.kron(np.eye(nsite), np.diag([1.0] * nv + [-1.0] * nv))


@pytest.fixture(scope="module")
def lvl():
    Lc1, nv1, nv2, agg2 = (6, 4, 2, 2), 3, 4, (2, 2, 1, 2)
    level1 = _random_level(Lc1, nv1, seed=3)
    W0 = synth.gaussian_coarse(Lc1, nv2, nv1, seed=3)
    P2 = amg.Prolongation(W0, Lc1, agg2)
    A2 = amg.coarse_operator(level1, P2)
    level2 = amg.CoarseLevel(A2, P2.Lc, nv2)
    return level1, P2, level2


def test_level2_lattice(lvl):
    level1, P2, level2 = lvl
    assert P2.Lc == (3, 2, 2, 1) and P2.asize == 8 and P2.d == 3
    assert level2.A.shape == (9, 1, 2, 2, 3, 8, 8)


def test_P2_orthonormal_and_chiral(lvl):
    level1, P2, level2 = lvl
    Pd = P2.dense()
    assert Pd.shape == (96 * 6, 12 * 8)
    assert np.abs(Pd.conj().T @ Pd - np.eye(Pd.shape[1])).max() < 1e-13
    assert np.abs(Pd.conj().T @ _g5c(96, 3) @ Pd - _g5c(12, 4)).max() < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.37])
def test_level2_is_galerkin(lvl, mu):
    # D_c2(mu) = P2^+ D_c1(mu) P2 exactly, the twisted mass included (P2 keeps gamma5_c)
    level1, P2, level2 = lvl
    Pd = P2.dense()
    ref = Pd.conj().T @ level1.dense(mu) @ Pd
    got = level2.dense(mu)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_level2_hops_are_nearest_neighbour(lvl):
    # on the 3-site x direction the forward and backward blocks differ and act on distinct sites
    level1, P2, level2 = lvl
    D = level2.dense(0.0).reshape(1, 2, 2, 3, 8, 1, 2, 2, 3, 8)
    # site (x=0) couples to x=1 through +x and to x=2 through -x; the two blocks are not equal
    fwd = D[0, 0, 0, 0, :, 0, 0, 0, 1, :]
    bwd = D[0, 0, 0, 0, :, 0, 0, 0, 2, :]
    assert np.abs(fwd).max() > 0.01 and np.abs(bwd).max() > 0.01
    assert np.abs(fwd - bwd).max() > 0.01
    assert np.allclose(fwd, level2.A[1, 0, 0, 0, 0]) and np.allclose(bwd, level2.A[2, 0, 0, 0, 0])


def test_mr_smooth_one_step_is_least_squares(lvl):
    level1, _, _ = lvl
    r = synth.gaussian_coarse(level1.L, 1, 3, seed=5)[0]
    e = amg.mr_smooth(level1, r, 0.2, 1)
    q = level1.apply(r, 0.2).ravel()
    c, *_ = np.linalg.lstsq(q[:, None], r.ravel(), rcond=None)
    assert np.abs(e.ravel() - c[0] * r.ravel()).max() < 1e-13 * np.abs(r).max()


def test_mr_smooth_residual_decreases(lvl):
    level1, _, _ = lvl
    r = synth.gaussian_coarse(level1.L, 1, 3, seed=6)[0]
    prev = np.linalg.norm(r)
    for k in range(1, 5):
        e = amg.mr_smooth(level1, r, 0.05, k)
        res = np.linalg.norm(r - level1.apply(e, 0.05))
        assert res < prev
        prev = res


def test_mr_smooth_exact_on_scaled_identity():
    Lc, nv = (2, 2, 2, 2), 2
    A = np.zeros((9,) + synth.lattice_shape(Lc) + (4, 4), dtype=np.complex128)
    A[0] = (2.5 - 0.5j) * np.eye(4)
    level = amg.CoarseLevel(A, Lc, nv)
    r = synth.gaussian_coarse(Lc, 1, nv, seed=7)[0]
    e = amg.mr_smooth(level, r, 0.0, 1)
    assert np.abs(e - r / (2.5 - 0.5j)).max() < 1e-14


def test_coarse_inverse_iteration_with_full_krylov_space():
    # gmres_steps = the level's dimension makes the approximate inverse exact
    Lc, nv = (2, 2, 2, 2), 2
    level = _random_level(Lc, nv, seed=8)
    W0 = synth.gaussian_coarse(Lc, 2, nv, seed=8)
    n = 16 * 4
    W = amg.setup_coarse_test_vectors(level, W0, 0.1, 1, n)
    D = level.dense(0.1)
    for k in range(2):
        x = np.linalg.solve(D, W0[k].ravel())
        x /= np.linalg.norm(x)
        assert np.abs(W[k].ravel() - x).max() < 1e-9


L4 = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def three():
    U = synth.gauge_field(L4, 0.3, seed=1)
    op = dirac.Operator(U, kappa=0.125, c_sw=1.0, bc_t=-1)
    V0 = synth.gaussian_spinors(L4, 8, seed=1, stream=301)
    W0 = synth.gaussian_coarse((2, 2, 2, 2), 6, 8, seed=1)
    mg = amg.ThreeLevelAMG(op, agg=(2, 2, 2, 2), V0=V0, sap_block=(2, 2, 2, 2), agg2=(1, 1, 2, 2), W0=W0,
                           setup_iters=2, setup_gmres_steps=10)
    return op, mg


def test_three_level_shapes(three):
    op, mg = three
    assert mg.P2.Lc == (2, 2, 1, 1) and mg.level2.A.shape == (9, 1, 1, 2, 2, 12, 12)


def test_three_level_cycle_reduces_to_two_level(three):
    # exact bottom solve and a middle FGMRES run to 1e-13: the cycle is the two-level cycle
    # with an exact coarse solve
    op, mg = three
    r = synth.gaussian_spinors(L4, 1, seed=9)[0]
    ref = mg.two.cycle(r, 0.01, coarse_mode="exact")
    got = mg.cycle(r, 0.01, mid_tol=1e-13, mid_restart=30, mid_maxiter=300, coarse_mode="exact")
    assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(ref)
    ex = mg.cycle(r, 0.01, mid_mode="exact")
    assert np.linalg.norm(ex - ref) < 1e-12 * np.linalg.norm(ref)


def test_three_level_solve_tiny(three):
    op, mg = three
    b = synth.gaussian_spinors(L4, 1, seed=10)[0]
    x, info = mg.solve(b, 0.01, tol=1e-10, restart=10)
    assert info["converged"] and info["resid"] <= 1e-10
    D = op.dense(0.01)
    xd = np.linalg.solve(D, b.ravel())
    assert np.linalg.norm(x.ravel() - xd) < 1e-7 * np.linalg.norm(xd)

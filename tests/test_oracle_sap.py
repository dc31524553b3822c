"""Pins for the oracle SAP smoother: block operator structure, MR, exactness limits."""
import numpy as np
import pytest

import synth
from oracle import dirac, sap


@pytest.fixture(scope="module")
def small():
    Ls = (4, 2, 2, 4)
    op = dirac.Operator(synth.gauge_field(Ls, 0.3, seed=21), kappa=0.11, c_sw=1.0)
    return Ls, op


def test_block_operator_is_masked_dense(small):
    # D_B equals D with every entry that couples two different blocks removed
    Ls, op = small
    bs = (2, 2, 1, 2)
    bop = sap.BlockOperator(op, bs)
    mu = 0.07
    M = op.dense(mu)
    bid, _ = sap.block_id(Ls, bs)
    site_block = np.repeat(bid.ravel(), 12)
    Mb = np.where(site_block[:, None] == site_block[None, :], M, 0)
    x = synth.gaussian_spinors(Ls, 1, seed=22)[0]
    assert np.abs(bop.apply(x, mu).ravel() - Mb @ x.ravel()).max() < 1e-13


def test_chessboard_colouring(small):
    Ls, op = small
    bs = (2, 1, 1, 2)
    col = sap.block_colour(Ls, bs)
    bc = sap.block_index(Ls, bs)
    # neighbouring blocks always have opposite colour (even block count per dimension)
    for ax, d in ((3, 0), (2, 1), (1, 2), (0, 3)):
        nb = np.roll(col, -bs[d], axis=ax)
        assert np.all(nb != col)
    assert set(np.unique(col)) == {0, 1}
    assert bc.shape[-1] == 4


def test_single_block_mr_converges_to_exact(small):
    # one block covering the lattice keeps every hop: D_B = D, so many MR steps solve D e = r
    Ls, op = small
    bop = sap.BlockOperator(op, Ls)
    r = synth.gaussian_spinors(Ls, 1, seed=23)[0]
    mu = 0.1
    e, rho = sap.mr_block_solve(bop, r, mu, 0, 400)
    x = np.linalg.solve(op.dense(mu), r.ravel())
    assert np.linalg.norm(e.ravel() - x) < 1e-9 * np.linalg.norm(x)
    assert np.linalg.norm(rho) < 1e-9 * np.linalg.norm(r)


def test_mr_residual_is_block_residual(small):
    # the returned rho is r_B - D_B e on the colour, zero elsewhere
    Ls, op = small
    bs = (2, 2, 1, 2)
    bop = sap.BlockOperator(op, bs)
    r = synth.gaussian_spinors(Ls, 1, seed=24)[0]
    mu = 0.02
    e, rho = sap.mr_block_solve(bop, r, mu, 1, 3)
    mask = (bop.colour == 1)[..., None, None]
    expect = (r - bop.apply(e, mu)) * mask
    assert np.abs(rho - expect).max() < 1e-13
    assert np.all(e[~np.broadcast_to(mask, e.shape)] == 0)


def test_sap_reduces_residual(small):
    Ls, op = small
    r = synth.gaussian_spinors(Ls, 2, seed=25)
    mu = np.array([0.01, 0.1])
    e = sap.sap(op, r, mu, (2, 2, 1, 2), cycles=3, mr_steps=4)
    res = r - op.apply(e, mu)
    for n in range(2):
        assert np.linalg.norm(res[n]) < 0.5 * np.linalg.norm(r[n])


def _dense_gauss_seidel(M, colour, r, cycles):
    """Multiplicative Schwarz with exact block solves, written with dense matrices: for each
    cycle, e_red += M_rr^{-1} (r - M e)_red, then e_black += M_bb^{-1} (r - M e)_black."""
    e = np.zeros_like(r)
    for _ in range(cycles):
        for c in (0, 1):
            sel = colour == c
            res = r - M @ e
            e[sel] += np.linalg.solve(M[np.ix_(sel, sel)], res[sel])
    return e


def test_sap_cycle_is_block_gauss_seidel(small):
    # Paper Sec. 2: SAP inverts the red blocks, then the black blocks on the residual that the red
    # correction left. On a 2 x 2 chessboard of blocks the two red blocks do not touch, so the red
    # block operator is the red-red part of D and one sweep with converged block solves is one step
    # of block Gauss-Seidel. Computing both colours from the same residual (additive Schwarz) or
    # reusing the red residual for the black sweep fails this pin.
    Ls = (4, 4, 2, 2)
    op = dirac.Operator(synth.gauge_field(Ls, 0.3, seed=26), kappa=0.11, c_sw=1.0)
    bs = (2, 2, 2, 2)
    mu = 0.05
    M = op.dense(mu)
    colour = np.repeat(sap.block_colour(Ls, bs).ravel(), 12)
    r = synth.gaussian_spinors(Ls, 1, seed=27)[0]
    for cycles in (1, 2):
        e = sap.sap(op, r, mu, bs, cycles=cycles, mr_steps=150)  # block MR converged (1e-15) well before 150
        ref = _dense_gauss_seidel(M, colour, r.ravel(), cycles)
        assert np.linalg.norm(e.ravel() - ref) < 1e-8 * np.linalg.norm(ref), cycles
    # the pin separates multiplicative from additive Schwarz on this lattice
    add = np.zeros_like(r.ravel())
    for c in (0, 1):
        sel = colour == c
        add[sel] = np.linalg.solve(M[np.ix_(sel, sel)], r.ravel()[sel])
    ref1 = _dense_gauss_seidel(M, colour, r.ravel(), 1)
    assert np.linalg.norm(add - ref1) > 1e-2 * np.linalg.norm(ref1)


def test_setup_test_vectors_is_inverse_power_iteration(small):
    # Paper Sec. 2: the test vectors approximate low modes by inverse iteration. With one SAP block
    # covering the lattice and its MR solve run to convergence, SAP(v) = D^{-1} v, so k setup steps
    # give D^{-k} v0 normalised (dense inverse power iteration).
    from oracle import amg
    Ls, op = small
    mu = 0.02
    V0 = synth.gaussian_spinors(Ls, 2, seed=28)
    k = 3
    V = amg.setup_test_vectors(op, V0, mu, Ls, k, sap_cycles=1, mr_steps=500)
    Minv = np.linalg.inv(op.dense(mu))
    for n in range(2):
        ref = V0[n].ravel()
        for _ in range(k):
            ref = Minv @ ref
        ref = ref / np.linalg.norm(ref)
        assert np.linalg.norm(V[n].ravel() - ref) < 1e-8, n
        assert abs(np.linalg.norm(V[n]) - 1.0) < 1e-12

"""Pins for the even-odd (Schur complement) oracle: dense block algebra on tiny lattices."""
import numpy as np
import pytest

import synth
from oracle import dirac, evenodd


@pytest.fixture(scope="module", params=[-1, 1])
def small(request):
    L = (4, 2, 2, 4)
    op = dirac.Operator(synth.gauge_field(L, 0.3, seed=71), kappa=0.125, c_sw=1.0, bc_t=request.param)
    return L, op


def _eo_index(L):
    par = evenodd.parity(L)
    ev = np.repeat((par == 0).ravel(), 12)
    return np.flatnonzero(ev), np.flatnonzero(~ev)


def test_hops_connect_opposite_parities(small):
    L, op = small
    par = evenodd.parity(L)
    x = synth.gaussian_spinors(L, 1, seed=72)[0]
    xe = np.where((par == 0)[..., None, None], x, 0)
    h = evenodd.apply_hops(op, xe)
    assert np.abs(h[par == 0]).max() == 0
    assert np.abs(h[par == 1]).max() > 0


def test_schur_complement_matches_dense_blocks(small):
    # M_ee = D_ee - D_eo D_oo^{-1} D_oe from the dense operator; a wrong sign of the correction term or
    # a missing local solve fails this
    L, op = small
    mu = 0.07
    D = op.dense(mu)
    e, o = _eo_index(L)
    M = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    x = synth.gaussian_spinors(L, 1, seed=73)[0]
    y = evenodd.schur_apply(op, x, mu)
    assert np.abs(y.ravel()[o]).max() == 0
    ref = M @ x.ravel()[e]
    assert np.linalg.norm(y.ravel()[e] - ref) < 1e-13 * np.linalg.norm(ref)


def test_schur_inverse_is_even_block_of_inverse(small):
    # (D^{-1})_ee = M_ee^{-1}: the reason the reduced system can be preconditioned by the full one
    L, op = small
    mu = -0.03
    D = op.dense(mu)
    e, o = _eo_index(L)
    M = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    Dinv = np.linalg.inv(D)
    assert np.linalg.norm(Dinv[np.ix_(e, e)] @ M - np.eye(len(e))) < 1e-10


def test_reduced_solve_solves_the_full_system(small):
    L, op = small
    mu = 0.02
    b = synth.gaussian_spinors(L, 1, seed=74)[0]
    x = evenodd.solve_via_schur(op, b, mu)
    ref = np.linalg.solve(op.dense(mu), b.ravel())
    assert np.linalg.norm(x.ravel() - ref) < 1e-10 * np.linalg.norm(ref)


def test_local_solve_inverts_the_site_blocks(small):
    L, op = small
    mu = 0.3
    x = synth.gaussian_spinors(L, 1, seed=75)[0]
    z = evenodd.local_solve(op, x, mu)
    back = op.apply_local(z) + op.apply_twist(z, mu)
    assert np.linalg.norm(back - x) < 1e-13 * np.linalg.norm(x)

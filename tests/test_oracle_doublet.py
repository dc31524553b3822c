"""Pins for the oracle's non-degenerate twisted-mass doublet operator."""
import numpy as np

import synth
from oracle import dirac, doublet
from oracle.gamma import gamma5, gammas


def test_zero_splitting_is_two_degenerate_operators():
    L = (4, 2, 2, 4)
    op = dirac.Operator(synth.gauge_field(L, 0.3, seed=31), kappa=0.12, c_sw=1.0)
    u, d = synth.gaussian_spinors(L, 2, seed=32)
    yu, yd = doublet.apply(op, u, d, 0.07, 0.0)
    assert np.abs(yu - op.apply(u, 0.07)).max() == 0
    assert np.abs(yd - op.apply(d, -0.07)).max() == 0


def test_gamma5_tau1_hermiticity():
    # (gamma5 tau1) D_ND (gamma5 tau1) = D_ND^+: tau1 swaps the flavours, tau1 tau3 tau1 = -tau3
    # turns the twist's sign and the splitting's tau1 is symmetric; a wrong sign of either term
    # or a flavour-diagonal splitting fails this
    L = (2, 2, 2, 4)
    op = dirac.Operator(synth.gauge_field(L, 0.3, seed=33), kappa=0.12, c_sw=1.0)
    M = doublet.dense(op, 0.11, 0.23)
    n = M.shape[0] // 2
    g5 = np.kron(np.eye(n // 12), np.kron(gamma5(), np.eye(3)))
    G = np.block([[np.zeros((n, n)), g5], [g5, np.zeros((n, n))]])
    assert np.abs(G @ M @ G - M.conj().T).max() < 1e-13


def test_free_field_plane_wave():
    # U = 1: on exp(i p.s) (u0, d0) the doublet acts as the 24 x 24 matrix
    # [[Dp(mu), -eps], [-eps, Dp(-mu)]] with Dp the free operator at momentum p
    Lf = (4, 2, 4, 8)
    kappa, mu, eps = 0.11, 0.3, 0.17
    op = dirac.Operator(synth.unit_gauge(Lf), kappa=kappa, c_sw=1.0, bc_t=-1)
    g = gammas()
    u0 = synth.complex_normal(3, 9, (4, 3))
    d0 = synth.complex_normal(4, 9, (4, 3))
    for n in [(0, 0, 0, 0), (1, 1, 3, 2), (3, 0, 1, 7)]:
        p = [2 * np.pi * n[k] / Lf[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / Lf[3]]
        t, z, y, x = np.meshgrid(*[np.arange(Lf[k]) for k in (3, 2, 1, 0)], indexing="ij")
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None, None]
        W = (1 / (2 * kappa) - sum(np.cos(pk) for pk in p)) * np.eye(4) + 1j * sum(g[k] * np.sin(p[k]) for k in range(4))
        Du = W + 1j * mu * gamma5()
        Dd = W - 1j * mu * gamma5()
        yu, yd = doublet.apply(op, phase * u0, phase * d0, mu, eps)
        assert np.abs(yu - phase * (Du @ u0 - eps * d0)).max() < 1e-13
        assert np.abs(yd - phase * (Dd @ d0 - eps * u0)).max() < 1e-13


def test_dense_matches_apply_and_is_invertible():
    L = (2, 2, 2, 4)
    op = dirac.Operator(synth.gauge_field(L, 0.3, seed=34), kappa=0.12, c_sw=1.0)
    M = doublet.dense(op, 0.05, 0.02)
    u, d = synth.gaussian_spinors(L, 2, seed=35)
    yu, yd = doublet.apply(op, u, d, 0.05, 0.02)
    assert np.abs(M @ np.concatenate([u.ravel(), d.ravel()]) - np.concatenate([yu.ravel(), yd.ravel()])).max() < 1e-13
    assert np.linalg.cond(M) < 1e4

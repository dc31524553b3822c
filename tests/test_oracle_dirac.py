"""Pins for the FP64 oracle operator D(mu) = D_W + c_sw C + i mu gamma5.

Each test checks the oracle against a fact fixed by the mathematics, not by
re-typing its own formula: gamma5-hermiticity, the twisted-mass normal-operator
identity, the free-field plane-wave closed form, gauge covariance, and a
constant abelian field whose clover term is known in closed form.
"""
import numpy as np
import pytest

import synth
from oracle import dirac
from oracle.gamma import gammas, gamma5

L = (4, 4, 2, 4)


def _inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


@pytest.fixture(scope="module")
def op():
    U = synth.gauge_field(L, 0.3, seed=11)
    return dirac.Operator(U, kappa=0.13, c_sw=1.0, bc_t=-1)


def test_gamma5_hermiticity(op):
    # gamma5 D(mu) gamma5 = D(-mu)^dagger  <=>  <y, g5 D(mu) g5 x> = <D(-mu) y, x>
    x, y = synth.gaussian_spinors(L, 2, seed=5)
    g5 = gamma5()
    mu = 0.37
    g5x = np.einsum("st,...tc->...sc", g5, x)
    lhs = _inner(y, np.einsum("st,...tc->...sc", g5, op.apply(g5x, mu)))
    rhs = _inner(op.apply(y, -mu), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_twisted_normal_identity(op):
    # D(mu)^dagger D(mu) = D(0)^dagger D(0) + mu^2
    x, y = synth.gaussian_spinors(L, 2, seed=6)
    mu = 0.21
    lhs = _inner(op.apply(x, mu), op.apply(y, mu))
    rhs = _inner(op.apply(x, 0.0), op.apply(y, 0.0)) + mu * mu * _inner(x, y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_twist_is_i_mu_gamma5(op):
    x = synth.gaussian_spinors(L, 1, seed=7)[0]
    mu = 0.05
    d = op.apply(x, mu) - op.apply(x, 0.0)
    assert np.allclose(d, 1j * mu * np.einsum("st,...tc->...sc", gamma5(), x), atol=1e-15)


@pytest.mark.parametrize("bc_t", [-1, 1])
def test_free_field_plane_wave(bc_t):
    # U = 1: D acting on exp(i p.s) u gives
    #   [1/(2 kappa) - sum cos p + i sum gamma sin p + i mu gamma5] u, with
    #   p_k = 2 pi n / L_k and p_t = (2 n + 1) pi / T for antiperiodic t.
    Lf = (4, 2, 4, 8)
    kappa, mu = 0.11, 0.3
    op = dirac.Operator(synth.unit_gauge(Lf), kappa=kappa, c_sw=1.0, bc_t=bc_t)
    g = gammas()
    rng_u = synth.complex_normal(3, 9, (4, 3))
    for n in [(0, 0, 0, 0), (1, 1, 3, 2), (3, 0, 1, 7)]:
        p = [2 * np.pi * n[k] / Lf[k] for k in range(3)]
        nt = n[3]
        p.append((2 * nt + (1 if bc_t == -1 else 0)) * np.pi / Lf[3])
        t, z, y, x = np.meshgrid(*[np.arange(Lf[d]) for d in (3, 2, 1, 0)], indexing="ij")
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * rng_u
        Dp = (1 / (2 * kappa) - sum(np.cos(pk) for pk in p)) * np.eye(4) \
            + 1j * sum(g[k] * np.sin(p[k]) for k in range(4)) + 1j * mu * gamma5()
        expect = phase[..., None, None] * (Dp @ rng_u)
        assert np.abs(op.apply(psi, mu) - expect).max() < 1e-13


def test_gauge_covariance(op):
    # U'_nu(s) = G(s) U_nu(s) G(s+nu)^dagger, x' = G x  =>  D[U'] x' = G D[U] x
    V = int(np.prod(L))
    G = synth.random_su3(V, seed=12).reshape((L[3], L[2], L[1], L[0], 3, 3))
    U = op.U
    Up = np.empty_like(U)
    for nu in range(4):
        disp = [1 if d == nu else 0 for d in range(4)]
        Gn = dirac.link_shift(G, disp)
        Up[..., nu, :, :] = G @ U[..., nu, :, :] @ dirac.dag(Gn)
    opp = dirac.Operator(Up, kappa=op.kappa, c_sw=op.c_sw, bc_t=op.bc_t)
    x = synth.gaussian_spinors(L, 1, seed=13)[0]
    Gx = np.einsum("...ab,...sb->...sa", G, x)
    mu = 0.1
    lhs = opp.apply(Gx, mu)
    rhs = np.einsum("...ab,...sb->...sa", G, op.apply(x, mu))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_clover_free_field_zero():
    C = dirac.clover_term(synth.unit_gauge(L), 1.0)
    assert np.abs(C).max() < 1e-15


def test_clover_hermitian_chiral(op):
    C = op.C
    assert np.abs(C - dirac.dag(C)).max() < 1e-14
    g5 = np.kron(gamma5(), np.eye(3))
    assert np.abs(C @ g5 - g5 @ C).max() < 1e-14
    assert np.abs(C).max() > 0.05


def test_clover_constant_abelian_field():
    # Constant U(1) field strength theta in the xy plane, embedded as phases times 1_3:
    # every xy plaquette is exp(i theta), all others 1. Then F_xy = i sin(theta) 1 and
    # C = -(c_sw/2) sin(theta) sigma_xy (x) 1_3 has eigenvalues +-(c_sw/2) sin(theta), six each.
    Lb = (4, 4, 2, 2)
    Lx, Ly = Lb[0], Lb[1]
    theta = 2 * np.pi / (Lx * Ly)
    U = synth.unit_gauge(Lb)
    t, z, y, x = np.meshgrid(*[np.arange(Lb[d]) for d in (3, 2, 1, 0)], indexing="ij")
    U[..., 1, :, :] *= np.exp(1j * theta * x)[..., None, None]
    edge = (x == Lx - 1)
    U[..., 0, :, :] *= np.where(edge, np.exp(-1j * theta * Lx * y), 1.0)[..., None, None]
    assert abs(dirac.plaquette(U) - (5 + np.cos(theta)) / 6) < 1e-14
    c_sw = 1.3
    C = dirac.clover_term(U, c_sw)
    ev = np.linalg.eigvalsh(C.reshape(-1, 12, 12))
    expect = np.array([-1] * 6 + [1] * 6) * 0.5 * c_sw * np.sin(theta)
    assert np.abs(ev - expect).max() < 1e-14


def test_dense_matches_apply(op):
    Ls = (2, 2, 2, 2)
    o = dirac.Operator(synth.gauge_field(Ls, 0.3, seed=2), 0.12, 1.0)
    M = o.dense(0.2)
    x = synth.gaussian_spinors(Ls, 1, seed=4)[0]
    assert np.abs(M @ x.ravel() - o.apply(x, 0.2).ravel()).max() < 1e-13

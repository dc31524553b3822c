"""Pins for the Dirac matrices: Clifford algebra, hermiticity, chirality."""
import numpy as np

from oracle.gamma import gammas, gamma5, sigma


def test_clifford_algebra():
    g = gammas()
    for mu in range(4):
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4), atol=1e-15)


def test_hermitian():
    for gm in gammas():
        assert np.allclose(gm, gm.conj().T)
    g5 = gamma5()
    assert np.allclose(g5, g5.conj().T)


def test_gamma5_chiral_and_anticommuting():
    g5 = gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    for gm in gammas():
        assert np.allclose(g5 @ gm + gm @ g5, 0)


def test_sigma_hermitian_commutes_with_gamma5():
    g5 = gamma5()
    for mu in range(4):
        for nu in range(4):
            s = sigma(mu, nu)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s @ g5, g5 @ s)
            assert np.allclose(s, -sigma(nu, mu))

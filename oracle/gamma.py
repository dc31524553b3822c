"""Euclidean Dirac matrices in a chiral basis (oracle; test infrastructure only).

The paper names no gamma basis. Reading taken: the chiral basis
  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3 for x, y, z)
  gamma_4 = [[0, 1], [1, 0]]                   (t)
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)
so that the clover term and i mu gamma_5 are block diagonal in chirality.
Pinned by the Clifford algebra and hermiticity (tests/test_oracle_gamma.py).
"""
import numpy as np

PAULI = np.array([
    [[0, 1], [1, 0]],
    [[0, -1j], [1j, 0]],
    [[1, 0], [0, -1]],
], dtype=np.complex128)

_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


def gammas():
    """gamma[0..3] for directions x, y, z, t; 4x4 complex."""
    g = [_block(_Z2, -1j * PAULI[k], 1j * PAULI[k], _Z2) for k in range(3)]
    g.append(_block(_Z2, _I2, _I2, _Z2))
    return np.array(g)


def gamma5():
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])

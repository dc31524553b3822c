"""Non-degenerate twisted-mass doublet in FP64 (oracle; test infrastructure only).

The paper (Sec. 1) notes that DDalphaAMG was adapted to degenerate twisted-mass fermions and then
generalised to the non-degenerate doublet. On a flavour doublet psi = (u, d) the operator is

    D_ND psi = ( D(mu) u - eps d ,  D(-mu) d - eps u )
             = D_W (x) 1 + i mu gamma5 (x) tau3 - eps 1 (x) tau1,

with D(mu) the degenerate operator of dirac.Operator (the same D_W: Wilson hops, clover, diagonal)
and eps >= 0 the mass splitting. Reading: this standard form (the paper gives no formula); the
twist enters with +mu on u and -mu on d, the splitting couples the flavours by -eps at every site
and spin-colour component. The multigrid hierarchy of the degenerate operator serves both
flavours unchanged: P and R act flavour by flavour, so the coarse doublet operator is
D_c(0) (x) 1 + i mu gamma5_c (x) tau3 - eps 1 (x) tau1.

Fields: u, d [..., T, Z, Y, X, 4, 3] with matching leading axes; mu and eps broadcast over them.
"""
import numpy as np

from . import dirac


def _bcast(a, x):
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(a.shape + (1,) * (x.ndim - a.ndim))


def apply(op: dirac.Operator, u, d, mu, eps):
    """(D(mu) u - eps d, D(-mu) d - eps u)."""
    mu = np.asarray(mu, dtype=np.float64)
    e = _bcast(eps, u)
    return op.apply(u, mu) - e * d, op.apply(d, -mu) - e * u


def dense(op: dirac.Operator, mu, eps):
    """The doublet operator as a dense (24 V) x (24 V) matrix [u block; d block] (tiny lattices)."""
    Du = op.dense(mu)
    Dd = op.dense(-mu)
    n = Du.shape[0]
    I = np.eye(n)
    return np.block([[Du, -eps * I], [-eps * I, Dd]])

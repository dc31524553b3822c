"""Even-odd (Schur complement) form of the twisted-mass Wilson-clover operator in FP64 (oracle; test
infrastructure only).

With the sites split by parity p(s) = (x + y + z + t) mod 2, the nearest-neighbour hops only connect
sites of opposite parity, so D(mu) = A(mu) + H has the block form

    D = [[A_ee, H_eo],
         [H_oe, A_oo]],

A(mu) the site-local part (diagonal 4 + m0, clover, i mu gamma5) and H the hop part. Eliminating the
odd sites leaves the Schur complement on the even sites

    M_ee = A_ee - H_eo A_oo^{-1} H_oe,

whose inverse is the even-even block of D^{-1}. The standard preconditioning of the (DD)alphaAMG
family: D x = b is solved as M_ee x_e = b_e - H_eo A_oo^{-1} b_o, then x_o = A_oo^{-1} (b_o - H_oe x_e).
The paper builds on that method family (Sec. 2) without restating this step; the formulas above are
the textbook Schur complement.

Fields: [..., T, Z, Y, X, 4, 3] as in dirac.Operator; mu broadcast over the leading axes.
"""
import numpy as np

from . import dirac


def parity(L):
    """Site parity [T, Z, Y, X] (0 even, 1 odd) of a lattice L = (Lx, Ly, Lz, Lt)."""
    t, z, y, x = np.meshgrid(np.arange(L[3]), np.arange(L[2]), np.arange(L[1]), np.arange(L[0]), indexing="ij")
    return (x + y + z + t) % 2


def _mask(x, par, p):
    """x with the sites of parity != p set to zero."""
    m = (par == p)[..., None, None]
    return np.where(m, x, 0)


def apply_hops(op: dirac.Operator, x):
    """H x: the eight hops of D (no local term)."""
    y = np.zeros_like(x)
    for nu in range(4):
        y = y + op.hop_fwd(x, nu) + op.hop_bwd(x, nu)
    return y


def local_matrices(op: dirac.Operator, mu):
    """A(mu) per site as 12 x 12 matrices [T, Z, Y, X, 12, 12] (spin-major, colour fastest)."""
    L = op.L
    n = 12
    A = np.zeros((L[3], L[2], L[1], L[0], n, n), dtype=np.complex128)
    eye = np.eye(n, dtype=np.complex128).reshape(n, 4, 3)
    for j in range(n):
        e = np.broadcast_to(eye[j], (L[3], L[2], L[1], L[0], 4, 3)).copy()
        A[..., :, j] = (op.apply_local(e) + op.apply_twist(e, mu)).reshape(L[3], L[2], L[1], L[0], n)
    return A


def local_solve(op: dirac.Operator, x, mu):
    """A(mu)^{-1} x site by site (one system: x [T, Z, Y, X, 4, 3], scalar mu)."""
    A = local_matrices(op, mu)
    shp = x.shape
    xf = x.reshape(shp[:-2] + (12,))
    return np.linalg.solve(A, xf[..., None])[..., 0].reshape(shp)


def schur_apply(op: dirac.Operator, x, mu):
    """M_ee x_e for the even part of x (its odd sites are ignored); the result is zero on odd sites.
    x [..., T, Z, Y, X, 4, 3] with leading system axes, mu broadcast over them."""
    par = parity(op.L)
    x = np.asarray(x)
    lead = x.shape[:-6]
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), lead)
    out = np.empty_like(x, dtype=np.complex128)
    for idx in np.ndindex(*lead):
        xe = _mask(x[idx], par, 0)
        t = _mask(apply_hops(op, xe), par, 1)              # H_oe x_e
        z = _mask(local_solve(op, t, float(mu[idx])), par, 1)  # A_oo^{-1} H_oe x_e
        y = op.apply_local(xe) + op.apply_twist(xe, float(mu[idx])) - apply_hops(op, z)
        out[idx] = _mask(y, par, 0)
    return out


def solve_via_schur(op: dirac.Operator, b, mu):
    """D(mu)^{-1} b through the even-odd reduction, the even system solved densely (tiny lattices)."""
    par = parity(op.L)
    be, bo = _mask(b, par, 0), _mask(b, par, 1)
    rhs = _mask(be - apply_hops(op, _mask(local_solve(op, bo, mu), par, 1)), par, 0)
    ev = np.repeat((par == 0).ravel(), 12)
    n = ev.sum()
    M = np.empty((n, n), dtype=np.complex128)
    shp = b.shape
    idx = np.flatnonzero(ev)
    for k, j in enumerate(idx):
        e = np.zeros(int(np.prod(shp)), dtype=np.complex128)
        e[j] = 1.0
        M[:, k] = schur_apply(op, e.reshape(shp), mu).ravel()[idx]
    xe = np.zeros(int(np.prod(shp)), dtype=np.complex128)
    xe[idx] = np.linalg.solve(M, rhs.ravel()[idx])
    xe = xe.reshape(shp)
    xo = _mask(local_solve(op, bo - _mask(apply_hops(op, xe), par, 1), mu), par, 1)
    return xe + xo

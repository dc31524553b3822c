"""Twisted-mass Wilson-clover operator in FP64 (oracle; test infrastructure only).

The operator (paper, Fig. 6 caption: D_TM = D_W + i (delta mu) mu gamma5, for
degenerate twisted-mass clover fermions, Sec. 1 / Sec. 2):

  D(mu) x(s) = (4 + m0) x(s) + c_sw C(s) x(s) + i mu gamma5 x(s)
               - 1/2 sum_nu [ (1 - gamma_nu) U_nu(s) x(s + nu)
                              + (1 + gamma_nu) U_nu(s - nu)^dagger x(s - nu) ]

Readings where the paper is silent:
  * m0 = 1/(2 kappa) - 4, so 4 + m0 = 1/(2 kappa);
  * mu enters in the same units as m0 (no 2 kappa factor);
  * C(s) = (i/4) sum_{mu,nu} sigma_{mu nu} (x) F_{mu nu}(s) with
    F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / 8 and Q the sum of the four
    clover-leaf plaquettes at s in the (mu, nu) plane; no trace subtraction;
  * boundary: periodic in x, y, z; phase bc_t (default -1, antiperiodic) on
    fermion hops that wrap in t. Gauge loops are periodic.

Array conventions: gauge field U [Lt, Lz, Ly, Lx, 4, 3, 3]; spinor fields
[..., Lt, Lz, Ly, Lx, 4, 3] (any leading batch axes). This module applies full
4x4 gamma matrices; it does not use spin projection or any other shortcut.
"""
import numpy as np

from .gamma import gammas, gamma5, sigma

# axis of direction nu in a spinor field [..., T, Z, Y, X, 4, 3]
_SPINOR_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}
# axis of direction nu in a link field [T, Z, Y, X, 3, 3]
_LINK_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}


def _bc_phase_fwd(shape, nu, bc_t, axis):
    """Phase multiplying x(s + nu): bc_t where s is on the last t slice."""
    if nu != 3 or bc_t == 1:
        return None
    L = shape[axis]
    ph = np.ones(L)
    ph[L - 1] = bc_t
    bshape = [1] * len(shape)
    bshape[axis] = L
    return ph.reshape(bshape)


def _bc_phase_bwd(shape, nu, bc_t, axis):
    """Phase multiplying x(s - nu): bc_t where s is on the first t slice."""
    if nu != 3 or bc_t == 1:
        return None
    L = shape[axis]
    ph = np.ones(L)
    ph[0] = bc_t
    bshape = [1] * len(shape)
    bshape[axis] = L
    return ph.reshape(bshape)


def shift_fwd(x, nu, bc_t=-1):
    """y(s) = x(s + nu) with the fermion boundary phase."""
    ax = _SPINOR_AXIS[nu]
    y = np.roll(x, -1, axis=ax)
    ph = _bc_phase_fwd(x.shape, nu, bc_t, ax)
    return y if ph is None else y * ph


def shift_bwd(x, nu, bc_t=-1):
    """y(s) = x(s - nu) with the fermion boundary phase."""
    ax = _SPINOR_AXIS[nu]
    y = np.roll(x, 1, axis=ax)
    ph = _bc_phase_bwd(x.shape, nu, bc_t, ax)
    return y if ph is None else y * ph


def link_shift(Unu, disp):
    """U(s + disp) for a single-direction link field [T, Z, Y, X, 3, 3]; periodic."""
    out = Unu
    for d, k in enumerate(disp):
        if k:
            out = np.roll(out, -k, axis=_LINK_AXIS[d])
    return out


def dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def clover_leaves(U, mu, nu):
    """Q_{mu nu}(s): sum of the four plaquettes in the (mu, nu) plane that start and end at s."""
    Umu = U[..., mu, :, :]
    Unu = U[..., nu, :, :]

    def e(d):
        v = [0, 0, 0, 0]
        for k, s in d:
            v[k] += s
        return v

    Umu_pnu = link_shift(Umu, e([(nu, 1)]))
    Unu_pmu = link_shift(Unu, e([(mu, 1)]))
    Umu_mmu = link_shift(Umu, e([(mu, -1)]))
    Unu_mmu = link_shift(Unu, e([(mu, -1)]))
    Umu_mmu_pnu = link_shift(Umu, e([(mu, -1), (nu, 1)]))
    Umu_mmu_mnu = link_shift(Umu, e([(mu, -1), (nu, -1)]))
    Unu_mmu_mnu = link_shift(Unu, e([(mu, -1), (nu, -1)]))
    Unu_mnu = link_shift(Unu, e([(nu, -1)]))
    Umu_mnu = link_shift(Umu, e([(nu, -1)]))
    Unu_pmu_mnu = link_shift(Unu, e([(mu, 1), (nu, -1)]))

    q1 = Umu @ Unu_pmu @ dag(Umu_pnu) @ dag(Unu)
    q2 = Unu @ dag(Umu_mmu_pnu) @ dag(Unu_mmu) @ Umu_mmu
    q3 = dag(Umu_mmu) @ dag(Unu_mmu_mnu) @ Umu_mmu_mnu @ Unu_mnu
    q4 = dag(Unu_mnu) @ Umu_mnu @ Unu_pmu_mnu @ dag(Umu)
    return q1 + q2 + q3 + q4


def field_strength(U, mu, nu):
    Q = clover_leaves(U, mu, nu)
    return (Q - dag(Q)) / 8.0


def clover_term(U, c_sw):
    """C(s) as a 12x12 matrix per site, index spin*3 + colour; Hermitian."""
    shape = U.shape[:4]
    C = np.zeros(shape + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = field_strength(U, mu, nu)
            s = sigma(mu, nu)
            C += np.einsum("ab,...ij->...aibj", s, F).reshape(shape + (12, 12))
    return c_sw * 0.25j * C


class Operator:
    """D(mu) = D_W + c_sw C + i mu gamma5 on one gauge field (FP64)."""

    def __init__(self, U, kappa, c_sw, bc_t=-1):
        self.U = np.asarray(U, dtype=np.complex128)
        self.kappa = float(kappa)
        self.c_sw = float(c_sw)
        self.bc_t = int(bc_t)
        self.L = (self.U.shape[3], self.U.shape[2], self.U.shape[1], self.U.shape[0])
        self.C = clover_term(self.U, self.c_sw)
        self.g = gammas()
        self.g5 = gamma5()
        self.eye4 = np.eye(4, dtype=np.complex128)
        # U_nu(s - nu)^dagger, precomputed per direction
        self.Ubwd = [dag(link_shift(self.U[..., nu, :, :], [(-1 if d == nu else 0) for d in range(4)]))
                     for nu in range(4)]

    @property
    def diag(self):
        """4 + m0 with m0 = 1/(2 kappa) - 4."""
        return 1.0 / (2.0 * self.kappa)

    def _spin(self, M, x):
        return np.einsum("st,...tc->...sc", M, x)

    def _col(self, Ulink, x):
        return np.einsum("...ab,...sb->...sa", Ulink, x)

    def hop_fwd(self, x, nu):
        """-1/2 (1 - gamma_nu) U_nu(s) x(s + nu)."""
        y = self._col(self.U[..., nu, :, :], shift_fwd(x, nu, self.bc_t))
        return -0.5 * self._spin(self.eye4 - self.g[nu], y)

    def hop_bwd(self, x, nu):
        """-1/2 (1 + gamma_nu) U_nu(s - nu)^dagger x(s - nu)."""
        y = self._col(self.Ubwd[nu], shift_bwd(x, nu, self.bc_t))
        return -0.5 * self._spin(self.eye4 + self.g[nu], y)

    def apply_clover(self, x):
        shp = x.shape
        xf = x.reshape(shp[:-2] + (12,))
        return np.einsum("...ij,...j->...i", self.C, xf).reshape(shp)

    def apply_local(self, x):
        """(4 + m0) x + c_sw C x (the site-diagonal part without the twist)."""
        return self.diag * x + self.apply_clover(x)

    def apply_twist(self, x, mu):
        """i mu gamma5 x; mu is a scalar or has the leading batch shape of x."""
        mu = np.asarray(mu, dtype=np.float64)
        mu = mu.reshape(mu.shape + (1,) * (x.ndim - mu.ndim))
        return 1j * mu * self._spin(self.g5, x)

    def apply(self, x, mu):
        """D(mu) x for x [..., T, Z, Y, X, 4, 3]; mu broadcast over the leading axes."""
        y = self.apply_local(x) + self.apply_twist(x, mu)
        for nu in range(4):
            y = y + self.hop_fwd(x, nu) + self.hop_bwd(x, nu)
        return y

    def apply_dagger(self, x, mu):
        """D(mu)^dagger x = gamma5 D(-mu) gamma5 x (gamma5-hermiticity, pinned in the tests)."""
        g5x = self._spin(self.g5, x)
        return self._spin(self.g5, self.apply(g5x, -np.asarray(mu)))

    def dense(self, mu):
        """The operator as a dense (12 V) x (12 V) matrix; tiny lattices only."""
        shp = self.U.shape[:4] + (4, 3)
        n = int(np.prod(shp))
        M = np.empty((n, n), dtype=np.complex128)
        chunk = 512
        for j0 in range(0, n, chunk):
            j1 = min(n, j0 + chunk)
            E = np.zeros((j1 - j0, n), dtype=np.complex128)
            E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
            M[:, j0:j1] = self.apply(E.reshape((j1 - j0,) + shp), mu).reshape(j1 - j0, n).T
        return M


def plaquette(U):
    """Average Re tr(plaquette)/3 over all sites and planes (a workload check)."""
    tot = 0.0
    cnt = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Umu = U[..., mu, :, :]
            Unu = U[..., nu, :, :]
            e_mu = [1 if d == mu else 0 for d in range(4)]
            e_nu = [1 if d == nu else 0 for d in range(4)]
            P = Umu @ link_shift(Unu, e_mu) @ dag(link_shift(Umu, e_nu)) @ dag(Unu)
            tot += np.trace(P, axis1=-2, axis2=-1).real.mean() / 3.0
            cnt += 1
    return tot / cnt

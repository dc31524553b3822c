"""Aggregation-based adaptive algebraic multigrid in FP64 (oracle; test infrastructure only).

Paper Sec. 2: prolongation P and restriction R = P^dagger are built from a few
approximate low modes ("test vectors", Luescher's inexact deflation) on
aggregates of the lattice; the coarse operator is D_c = P^dagger D P on the
coarse lattice of aggregates; the construction recurses to further levels.
Paper Sec. 4 / Fig. 6 caption: on coarse levels the twisted mass enters as
i (delta mu) mu gamma5_c.

Readings where the paper is silent:
  * aggregates are rectangular blocks; every test vector is split by
    chirality (spins 0,1 versus 2,3 on the fine level; the first and second
    half of the coarse index on coarse levels), so a coarse site carries
    2 Nv unknowns and P^dagger gamma5 P = gamma5_c exactly;
  * per aggregate and chirality the Nv pieces are orthonormalised by
    classical Gram-Schmidt applied twice;
  * test vectors: start vectors (an input) smoothed by `setup_iters` steps of
    inverse iteration v <- SAP(v) / ||SAP(v)|| at mu = mu_setup;
  * AMG cycle: e = P D_c^{-1} P^dagger r, then e += SAP(r - D e) (SAP as a
    post-smoother only); the coarse system is solved by FGMRES to a relative
    residual (1e-1 at the bottom, the paper's tuned r_b), by block GMRES, or exactly;
  * three levels: the level-2 test vectors are smoothed by inverse iteration with
    a fixed number of level-1 GMRES steps; the middle level is solved by FGMRES to
    r_m preconditioned by the level-2 correction plus a few minimal-residual steps
    on the level-1 residual (the paper names no coarse-level smoother).

Field layout used here: a level's vector is [..., T, Z, Y, X, 2, d] with the
chirality axis (2) and d unknowns per chirality (d = 6 = 2 spins x 3 colours
on the fine level). Coarse site order is lexicographic, x fastest.
"""
import numpy as np

from . import dirac, sap as sap_mod, krylov

# hop index convention for the coarse stencil: 0 = self, 1 + 2 nu = +nu, 2 + 2 nu = -nu
NHOP = 9


def hop_index(nu, sign):
    return 1 + 2 * nu + (0 if sign > 0 else 1)


def coarse_extent(L, agg):
    for d in range(4):
        if L[d] % agg[d]:
            raise ValueError("aggregate extent must divide the lattice extent")
    return tuple(L[d] // agg[d] for d in range(4))


def to_agg(f, L, agg, ntrail):
    """lead + (T, Z, Y, X) + trail  ->  lead + (Vc, |a|) + trail (|a| ordered x fastest)."""
    Lx, Ly, Lz, Lt = L
    ax, ay, az, at = agg
    lead = f.shape[:f.ndim - 4 - ntrail]
    trail = f.shape[f.ndim - ntrail:]
    nl = len(lead)
    g = f.reshape(lead + (Lt // at, at, Lz // az, az, Ly // ay, ay, Lx // ax, ax) + trail)
    perm = list(range(nl)) + [nl + 0, nl + 2, nl + 4, nl + 6, nl + 1, nl + 3, nl + 5, nl + 7] + \
        list(range(nl + 8, nl + 8 + ntrail))
    g = g.transpose(perm)
    Vc = (Lt // at) * (Lz // az) * (Ly // ay) * (Lx // ax)
    return g.reshape(lead + (Vc, at * az * ay * ax) + trail)


def from_agg(g, L, agg, ntrail):
    """Inverse of to_agg."""
    Lx, Ly, Lz, Lt = L
    ax, ay, az, at = agg
    lead = g.shape[:g.ndim - 2 - ntrail]
    trail = g.shape[g.ndim - ntrail:]
    nl = len(lead)
    h = g.reshape(lead + (Lt // at, Lz // az, Ly // ay, Lx // ax, at, az, ay, ax) + trail)
    perm = list(range(nl)) + [nl + 0, nl + 4, nl + 1, nl + 5, nl + 2, nl + 6, nl + 3, nl + 7] + \
        list(range(nl + 8, nl + 8 + ntrail))
    h = h.transpose(perm)
    return h.reshape(lead + (Lt, Lz, Ly, Lx) + trail)


def orthonormalise(X):
    """Columns of X [..., m, k] made orthonormal by classical Gram-Schmidt, applied twice."""
    Q = np.array(X, dtype=np.complex128)
    k = Q.shape[-1]
    for j in range(k):
        w = Q[..., j]
        for _ in range(2):
            if j > 0:
                Qj = Q[..., :j]
                c = np.einsum("...mi,...m->...i", np.conj(Qj), w)
                w = w - np.einsum("...mi,...i->...m", Qj, c)
        nrm = np.linalg.norm(w, axis=-1, keepdims=True)
        Q[..., j] = w / nrm
    return Q


class Prolongation:
    """P for one level: per aggregate and chirality an orthonormal (|a| d) x Nv block."""

    def __init__(self, V, L, agg):
        # V: test vectors [Nv, T, Z, Y, X, 2, d]
        self.L = tuple(L)
        self.agg = tuple(agg)
        self.Lc = coarse_extent(L, agg)
        self.Nv = V.shape[0]
        self.d = V.shape[-1]
        Va = to_agg(V, L, agg, 2)                  # [Nv, Vc, |a|, 2, d]
        self.asize = Va.shape[2]
        X = Va.transpose(1, 3, 2, 4, 0)            # [Vc, 2, |a|, d, Nv]
        Vc = X.shape[0]
        X = X.reshape(Vc, 2, self.asize * self.d, self.Nv)
        self.Q = orthonormalise(X)                 # [Vc, 2, |a| d, Nv]

    @property
    def nc(self):
        return 2 * self.Nv

    def restrict(self, r):
        """r: lead + (T, Z, Y, X, 2, d)  ->  lead + (Tc, Zc, Yc, Xc, 2, Nv)."""
        ra = to_agg(r, self.L, self.agg, 2)          # lead + (Vc, |a|, 2, d)
        ra = np.moveaxis(ra, -3, -2)                  # lead + (Vc, 2, |a|, d)
        ra = ra.reshape(ra.shape[:-2] + (self.asize * self.d,))
        xc = np.einsum("ckmj,...ckm->...ckj", np.conj(self.Q), ra)  # lead + (Vc, 2, Nv)
        Lxc, Lyc, Lzc, Ltc = self.Lc
        return xc.reshape(xc.shape[:-3] + (Ltc, Lzc, Lyc, Lxc, 2, self.Nv))

    def prolong(self, xc):
        """lead + (Tc, Zc, Yc, Xc, 2, Nv)  ->  lead + (T, Z, Y, X, 2, d)."""
        lead = xc.shape[:-6]
        xcf = xc.reshape(lead + (-1, 2, self.Nv))
        e = np.einsum("ckmj,...ckj->...ckm", self.Q, xcf)  # lead + (Vc, 2, |a| d)
        e = e.reshape(lead + (e.shape[-3], 2, self.asize, self.d))
        e = np.moveaxis(e, -3, -2)                          # lead + (Vc, |a|, 2, d)
        return from_agg(e, self.L, self.agg, 2)

    def dense(self):
        """P as a dense (V 2 d) x (Vc 2 Nv) matrix (tiny lattices only)."""
        Vc = self.Q.shape[0]
        n_c = Vc * 2 * self.Nv
        cols = []
        for a in range(Vc):
            for chi in range(2):
                for j in range(self.Nv):
                    xc = np.zeros((Vc, 2, self.Nv), dtype=np.complex128)
                    xc[a, chi, j] = 1.0
                    Lxc, Lyc, Lzc, Ltc = self.Lc
                    cols.append(self.prolong(xc.reshape(Ltc, Lzc, Lyc, Lxc, 2, self.Nv)).ravel())
        M = np.array(cols).T
        assert M.shape[1] == n_c
        return M


class FineLevel:
    """The fine operator seen through the level interface: vectors [..., T, Z, Y, X, 2, 6]."""

    def __init__(self, op: dirac.Operator):
        self.op = op
        self.L = op.L
        self.d = 6

    @staticmethod
    def to_spin(x):
        return x.reshape(x.shape[:-2] + (4, 3))

    @staticmethod
    def to_chi(x):
        return x.reshape(x.shape[:-2] + (2, 6))

    def local(self, x):
        return self.to_chi(self.op.apply_local(self.to_spin(x)))

    def hop(self, x, nu, sign):
        xs = self.to_spin(x)
        y = self.op.hop_fwd(xs, nu) if sign > 0 else self.op.hop_bwd(xs, nu)
        return self.to_chi(y)

    def twist(self, x, mu):
        return self.to_chi(self.op.apply_twist(self.to_spin(x), mu))

    def apply(self, x, mu):
        return self.to_chi(self.op.apply(self.to_spin(x), mu))


_COARSE_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}


class CoarseLevel:
    """Coarse 9-point operator y(a) = sum_h A_h(a) x(a + h) + i mu gamma5_c x(a).

    A: [9, Tc, Zc, Yc, Xc, n_c, n_c]; vectors [..., Tc, Zc, Yc, Xc, 2, Nv].
    Coarse hops are periodic: the fermion boundary phase is already inside A.
    """

    def __init__(self, A, Lc, Nv):
        self.A = A
        self.L = tuple(Lc)
        self.Nv = Nv
        self.d = Nv

    def _mat(self, h, x):
        xf = x.reshape(x.shape[:-2] + (2 * self.Nv,))
        y = np.einsum("...ij,...j->...i", self.A[h], xf)
        return y.reshape(x.shape)

    def local(self, x):
        return self._mat(0, x)

    def hop(self, x, nu, sign):
        ax = _COARSE_AXIS[nu]
        xs = np.roll(x, -1 if sign > 0 else 1, axis=ax)
        return self._mat(hop_index(nu, sign), xs)

    def twist(self, x, mu):
        mu = np.asarray(mu, dtype=np.float64)
        mu = mu.reshape(mu.shape + (1,) * (x.ndim - mu.ndim))
        g5 = np.array([1.0, -1.0]).reshape(2, 1)
        return 1j * mu * g5 * x

    def apply(self, x, mu):
        y = self.local(x) + self.twist(x, mu)
        for nu in range(4):
            y = y + self.hop(x, nu, +1) + self.hop(x, nu, -1)
        return y

    def dense(self, mu):
        Lxc, Lyc, Lzc, Ltc = self.L
        n = Ltc * Lzc * Lyc * Lxc * 2 * self.Nv
        E = np.eye(n, dtype=np.complex128).reshape((n, Ltc, Lzc, Lyc, Lxc, 2, self.Nv))
        return self.apply(E, mu).reshape(n, n).T


def coarse_operator(level, P: Prolongation, chunk=16):
    """A_h(a)[i, j] = < P_i on a , (part h of D) P_j on a + h >, for the 9 hop classes h.

    A hop of the fine operator whose two ends lie in the same aggregate belongs
    to the self block; one that crosses into the neighbouring aggregate in
    direction h belongs to A_h. The twisted mass is left out (added as
    i mu gamma5_c on the coarse level).
    """
    L = level.L
    agg = P.agg
    Lc = P.Lc
    Nv = P.Nv
    n_c = 2 * Nv
    Vc = int(np.prod(Lc))
    # aggregate id of every fine site, and of its neighbours
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    coords = [x, y, z, t]
    aid = ((t // agg[3] * Lc[2] + z // agg[2]) * Lc[1] + y // agg[1]) * Lc[0] + x // agg[0]
    site_axis = {0: 3, 1: 2, 2: 1, 3: 0}
    A = np.zeros((NHOP, Vc, n_c, n_c), dtype=np.complex128)
    # column j of P over all aggregates at once
    cols = list(range(n_c))
    for c0 in range(0, n_c, chunk):
        cs = cols[c0:c0 + chunk]
        xc = np.zeros((len(cs), Vc, 2, Nv), dtype=np.complex128)
        for k, c in enumerate(cs):
            xc[k, :, c // Nv, c % Nv] = 1.0
        Lxc, Lyc, Lzc, Ltc = Lc
        W = P.prolong(xc.reshape(len(cs), Ltc, Lzc, Lyc, Lxc, 2, Nv))  # [k, T, Z, Y, X, 2, d]
        self_part = level.local(W)
        for nu in range(4):
            for sign in (+1, -1):
                nb = np.roll(aid, -sign, axis=site_axis[nu])
                inside = (nb == aid).astype(np.float64)[..., None, None]
                hp = level.hop(W, nu, sign)
                self_part = self_part + inside * hp
                cross = (1.0 - inside) * hp
                rc = P.restrict(cross).reshape(len(cs), Vc, n_c)
                A[hop_index(nu, sign), :, :, c0:c0 + len(cs)] = np.moveaxis(rc, 0, -1)
        rc = P.restrict(self_part).reshape(len(cs), Vc, n_c)
        A[0, :, :, c0:c0 + len(cs)] = np.moveaxis(rc, 0, -1)
    del coords
    Lxc, Lyc, Lzc, Ltc = Lc
    return A.reshape((NHOP, Ltc, Lzc, Lyc, Lxc, n_c, n_c))


def setup_test_vectors(op: dirac.Operator, V0, mu_setup, sap_block, setup_iters, sap_cycles=2, mr_steps=3):
    """Inverse iteration v <- SAP(v)/||SAP(v)|| on the start vectors V0 [Nv, T, Z, Y, X, 4, 3]."""
    V = np.array(V0, dtype=np.complex128)
    bop = sap_mod.BlockOperator(op, sap_block)
    mus = np.full(V.shape[0], mu_setup)
    for _ in range(setup_iters):
        V = sap_mod.sap(op, V, mus, sap_block, cycles=sap_cycles, mr_steps=mr_steps, bop=bop)
        nrm = np.sqrt(np.sum(np.abs(V) ** 2, axis=tuple(range(1, V.ndim))))
        V = V / nrm.reshape((-1,) + (1,) * (V.ndim - 1))
    return V


class TwoLevelAMG:
    """Fine level + one coarse level (the method's 2-level configuration)."""

    def __init__(self, op: dirac.Operator, agg, V0, sap_block, setup_iters=5, mu_setup=0.0,
                 sap_cycles=2, mr_steps=3, delta_mu=1.0):
        self.op = op
        self.fine = FineLevel(op)
        self.sap_block = tuple(sap_block)
        self.sap_cycles = sap_cycles
        self.mr_steps = mr_steps
        self.delta_mu = delta_mu
        self.bop = sap_mod.BlockOperator(op, sap_block)
        V = setup_test_vectors(op, V0, mu_setup, sap_block, setup_iters, sap_cycles, mr_steps)
        self.V = V
        self.P = Prolongation(FineLevel.to_chi(V), op.L, agg)
        self.A = coarse_operator(self.fine, self.P)
        self.coarse = CoarseLevel(self.A, self.P.Lc, self.P.Nv)

    def coarse_solve(self, rc, mu_c, mode, tol, restart, maxiter):
        shp = rc.shape
        if mode == "exact":
            M = self.coarse.dense(mu_c)
            return np.linalg.solve(M, rc.ravel()).reshape(shp)
        A = lambda v: self.coarse.apply(v.reshape(shp), mu_c).ravel()
        x, _ = krylov.fgmres(A, rc.ravel(), tol=tol, restart=restart, maxiter=maxiter)
        return x.reshape(shp)

    def cycle(self, r, mu, coarse_mode="fgmres", coarse_tol=1e-1, coarse_restart=20, coarse_maxiter=200,
              smooth=True):
        """One AMG cycle on a single fine vector r [T, Z, Y, X, 4, 3] at twisted mass mu."""
        rc = self.P.restrict(FineLevel.to_chi(r))
        ec = self.coarse_solve(rc, self.delta_mu * mu, coarse_mode, coarse_tol, coarse_restart, coarse_maxiter)
        e = FineLevel.to_spin(self.P.prolong(ec))
        if smooth:
            r2 = r - self.op.apply(e, mu)
            e = e + sap_mod.sap(self.op, r2, mu, self.sap_block, self.sap_cycles, self.mr_steps, bop=self.bop)
        return e

    def solve(self, b, mu, tol=1e-10, restart=10, maxiter=500, **cycle_kw):
        """FGMRES(restart) preconditioned by one AMG cycle; one rhs, one shift."""
        shp = b.shape
        A = lambda v: self.op.apply(v.reshape(shp), mu).ravel()
        M = lambda v: self.cycle(v.reshape(shp), mu, **cycle_kw).ravel()
        x, info = krylov.fgmres(A, b.ravel(), tol=tol, restart=restart, maxiter=maxiter, M=M)
        return x.reshape(shp), info


# ---------------------------------------------------------------------------------------------
# Three levels (paper Sec. 4: a three-level AMG with FGMRES at the top; the middle level is
# solved by FGMRES to r_m, about 7e-2, the bottom to r_b, about 1e-1; Sec. 2: the construction
# is applied recursively to the coarse lattice).

def mr_smooth(level, r, mu, steps):
    """`steps` minimal-residual steps on `level` from a zero start: with q = D rho,
    alpha = <q, rho> / <q, q>, e += alpha rho, rho -= alpha q (each step minimises |rho - alpha q|).

    Reading: the paper names no smoother for the coarse levels; the middle level's cycle uses
    these few global MR steps as its post-smoother."""
    e = np.zeros_like(r, dtype=np.complex128)
    rho = np.array(r, dtype=np.complex128)
    for _ in range(steps):
        q = level.apply(rho, mu)
        qq = np.vdot(q, q).real
        if qq == 0.0:
            break
        alpha = np.vdot(q, rho) / qq
        e = e + alpha * rho
        rho = rho - alpha * q
    return e


def setup_coarse_test_vectors(level, W0, mu_setup, setup_iters, gmres_steps):
    """Inverse iteration on a coarse level, w <- G(w) / |G(w)|, where G is `gmres_steps` Arnoldi
    steps of GMRES on D_c(mu_setup) from a zero start (the level's approximate inverse; the
    fine level uses SAP in this role). W0: [Nv, Tc, Zc, Yc, Xc, 2, d]."""
    W = np.array(W0, dtype=np.complex128)
    shp = W.shape[1:]
    A = lambda v: level.apply(v.reshape(shp), mu_setup).ravel()
    for _ in range(setup_iters):
        for k in range(W.shape[0]):
            x, _ = krylov.fgmres(A, W[k].ravel(), tol=0.0, restart=gmres_steps, maxiter=gmres_steps)
            W[k] = (x / np.linalg.norm(x)).reshape(shp)
    return W


class ThreeLevelAMG:
    """Fine level + two coarse levels.

    Level 1 is built as in TwoLevelAMG. Level 2 aggregates the level-1 lattice (agg2) with Nv2
    test vectors W0 on level 1 (split by the chirality of gamma5_c), smoothed by inverse iteration
    with level-1 GMRES; D_c2 = P2^+ D_c1 P2 on its hop classes. The AMG cycle is
        e = P1 x1,  x1 ~ D_c1^{-1} P1^+ r  by FGMRES on level 1 to mid_tol, preconditioned by
            z = P2 x2 with x2 ~ D_c2^{-1} P2^+ v (GMRES to coarse_tol), then z += MR(v - D_c1 z);
        e += SAP(r - D e).
    Twisted mass on both coarse levels: i (delta mu) mu gamma5_c.
    """

    def __init__(self, op: dirac.Operator, agg, V0, sap_block, agg2, W0, setup_iters=5, mu_setup=0.0,
                 sap_cycles=2, mr_steps=3, delta_mu=1.0, setup_gmres_steps=20, mid_smooth=3):
        self.two = TwoLevelAMG(op, agg, V0, sap_block, setup_iters, mu_setup, sap_cycles, mr_steps, delta_mu)
        self.op = op
        self.delta_mu = delta_mu
        self.P1 = self.two.P
        self.level1 = self.two.coarse
        self.W = setup_coarse_test_vectors(self.level1, W0, mu_setup, setup_iters, setup_gmres_steps)
        self.P2 = Prolongation(self.W, self.level1.L, agg2)
        self.A2 = coarse_operator(self.level1, self.P2)
        self.level2 = CoarseLevel(self.A2, self.P2.Lc, self.P2.Nv)
        self.mid_smooth = mid_smooth

    def bottom_solve(self, rc, mu_c, mode, tol, restart, maxiter):
        shp = rc.shape
        if mode == "exact":
            return np.linalg.solve(self.level2.dense(mu_c), rc.ravel()).reshape(shp)
        A = lambda v: self.level2.apply(v.reshape(shp), mu_c).ravel()
        x, _ = krylov.fgmres(A, rc.ravel(), tol=tol, restart=restart, maxiter=maxiter)
        return x.reshape(shp)

    def mid_cycle(self, v, mu_c, coarse_mode="fgmres", coarse_tol=1e-1, coarse_restart=20, coarse_maxiter=200):
        """Preconditioner of the middle FGMRES: level-2 correction, then MR post-smoothing."""
        x2 = self.bottom_solve(self.P2.restrict(v), mu_c, coarse_mode, coarse_tol, coarse_restart, coarse_maxiter)
        z = self.P2.prolong(x2)
        if self.mid_smooth:
            z = z + mr_smooth(self.level1, v - self.level1.apply(z, mu_c), mu_c, self.mid_smooth)
        return z

    def mid_solve(self, rc, mu_c, mid_mode="fgmres", mid_tol=7e-2, mid_restart=10, mid_maxiter=50, **bottom):
        shp = rc.shape
        if mid_mode == "exact":
            return np.linalg.solve(self.level1.dense(mu_c), rc.ravel()).reshape(shp)
        A = lambda v: self.level1.apply(v.reshape(shp), mu_c).ravel()
        M = lambda v: self.mid_cycle(v.reshape(shp), mu_c, **bottom).ravel()
        x, _ = krylov.fgmres(A, rc.ravel(), tol=mid_tol, restart=mid_restart, maxiter=mid_maxiter, M=M)
        return x.reshape(shp)

    def cycle(self, r, mu, smooth=True, **kw):
        """One AMG cycle on a single fine vector r [T, Z, Y, X, 4, 3] at twisted mass mu."""
        rc = self.P1.restrict(FineLevel.to_chi(r))
        ec = self.mid_solve(rc, self.delta_mu * mu, **kw)
        e = FineLevel.to_spin(self.P1.prolong(ec))
        if smooth:
            r2 = r - self.op.apply(e, mu)
            two = self.two
            e = e + sap_mod.sap(self.op, r2, mu, two.sap_block, two.sap_cycles, two.mr_steps, bop=two.bop)
        return e

    def solve(self, b, mu, tol=1e-10, restart=10, maxiter=500, **cycle_kw):
        """FGMRES(restart) preconditioned by one three-level AMG cycle; one rhs, one shift."""
        shp = b.shape
        A = lambda v: self.op.apply(v.reshape(shp), mu).ravel()
        M = lambda v: self.cycle(v.reshape(shp), mu, **cycle_kw).ravel()
        x, info = krylov.fgmres(A, b.ravel(), tol=tol, restart=restart, maxiter=maxiter, M=M)
        return x.reshape(shp), info

"""GPU parity of the second coarse level (P2^+, P2, D_c2 = P2^+ D_c1 P2) against the FP64 oracle
built from the same injected test vectors, the middle and bottom coarse solves of a three-level
hierarchy checked by the oracle's level operators, and end-to-end three-level solves checked by
the oracle's fine operator.

Tolerances: D_c1 is built in FP32 (relative error about 1e-7), P2 by FP32 Gram-Schmidt with FP64
dots, and D_c2 from FP32 hop parts and restrictions; 2e-5 covers that chain as for level 1."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac
from tests.gpu_util import Lattice, coarse_from_bundle, coarse_to_bundle, relerr
from tests.test_gpu_amg import _f16_bound

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _setup3(L, agg, nv, agg2, nv2, seed=91):
    U = synth.gauge_field(L, 0.3, seed=seed)
    lat = Lattice(L, U, 0.125, 1.0)
    T = lat.T
    Vt = synth.gaussian_spinors(L, nv, seed=seed + 1).astype(np.complex64)
    Lc1 = amg.coarse_extent(L, agg)
    W0 = synth.gaussian_coarse(Lc1, nv2, nv, seed=seed + 2).astype(np.complex64)
    vecs = np.concatenate([Vt.ravel(), W0.ravel()])
    p = T.setup_params(levels=3, agg=agg, nv=nv, sap_block=(2, 2, 2, 2), setup_iters=0, agg2=agg2, nv2=nv2)
    dev = lat.torch.from_numpy(vecs.view(np.float32).copy()).cuda()
    T.tmamg_setup_from_vectors(lat.ctx, p, dev)
    op = dirac.Operator(U, 0.125, 1.0)
    P1 = amg.Prolongation(amg.FineLevel.to_chi(Vt.astype(np.complex128)), L, agg)
    level1 = amg.CoarseLevel(amg.coarse_operator(amg.FineLevel(op), P1), P1.Lc, nv)
    P2 = amg.Prolongation(W0.astype(np.complex128), Lc1, agg2)
    level2 = amg.CoarseLevel(amg.coarse_operator(level1, P2), P2.Lc, nv2)
    return lat, level1, P2, level2


CASES = [((8, 8, 8, 8), (2, 2, 2, 2), 6, (2, 2, 2, 2), 8),
         ((12, 8, 8, 8), (2, 2, 2, 2), 6, (2, 2, 2, 2), 10),
         ((8, 4, 4, 8), (2, 2, 2, 2), 8, (1, 2, 2, 2), 12)]


@pytest.mark.parametrize("L,agg,nv,agg2,nv2", CASES)
def test_level2_restrict_prolong_match_oracle(L, agg, nv, agg2, nv2):
    lat, level1, P2, level2 = _setup3(L, agg, nv, agg2, nv2)
    try:
        nsys = 3
        Vc1, Vc2 = int(np.prod(level1.L)), int(np.prod(P2.Lc))
        nc1, nc2 = 2 * nv, 2 * nv2
        shp1 = synth.lattice_shape(level1.L) + (2, nv)
        shp2 = synth.lattice_shape(P2.Lc) + (2, nv2)
        x1 = synth.complex_normal(93, 1, (nsys, Vc1, nc1))
        xb = lat.torch.from_numpy(coarse_to_bundle(x1, nc1, Vc1)).cuda()
        cb = lat.coarse_buffer(nsys, level=2)
        lat.T.tmamg_restrict(lat.ctx, 2, xb, cb, nsys)
        lat.torch.cuda.synchronize()
        got = coarse_from_bundle(cb.cpu().numpy(), nsys, nc2, Vc2)
        ref = P2.restrict(x1.reshape((nsys,) + shp1)).reshape(nsys, Vc2, nc2)
        for n in range(nsys):
            assert relerr(got[n], ref[n]) < TOL32, (n, relerr(got[n], ref[n]))
        y2 = synth.complex_normal(94, 1, (nsys, Vc2, nc2))
        yb = lat.torch.from_numpy(coarse_to_bundle(y2, nc2, Vc2)).cuda()
        pb = lat.coarse_buffer(nsys, level=1)
        lat.T.tmamg_prolong(lat.ctx, 2, yb, pb, nsys)
        lat.torch.cuda.synchronize()
        got = coarse_from_bundle(pb.cpu().numpy(), nsys, nc1, Vc1)
        ref = P2.prolong(y2.reshape((nsys,) + shp2)).reshape(nsys, Vc1, nc1)
        for n in range(nsys):
            assert relerr(got[n], ref[n]) < TOL32, (n, relerr(got[n], ref[n]))
    finally:
        lat.close()


@pytest.mark.parametrize("L,agg,nv,agg2,nv2", CASES)
def test_level2_operator_matches_oracle(L, agg, nv, agg2, nv2):
    lat, level1, P2, level2 = _setup3(L, agg, nv, agg2, nv2)
    try:
        nsys = 5
        Vc2, nc2 = int(np.prod(P2.Lc)), 2 * nv2
        shp2 = synth.lattice_shape(P2.Lc) + (2, nv2)
        x = synth.complex_normal(95, 1, (nsys, Vc2, nc2))
        mu = np.linspace(-0.1, 0.3, nsys)
        xb = lat.torch.from_numpy(coarse_to_bundle(x, nc2, Vc2)).cuda()
        ref = level2.apply(x.reshape((nsys,) + shp2), mu).reshape(nsys, Vc2, nc2)
        yb = lat.coarse_buffer(nsys, level=2)
        lat.T.tmamg_coarse_apply(lat.ctx, 2, xb, yb, nsys, mu, 32)
        lat.torch.cuda.synchronize()
        y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc2, Vc2)
        for n in range(nsys):
            assert relerr(y[n], ref[n]) < TOL32, (n, relerr(y[n], ref[n]))
        # the FP16 tensor-core stencil on level 2, within its elementwise bound
        yb.zero_()
        lat.T.tmamg_coarse_apply(lat.ctx, 2, xb, yb, nsys, mu, 16)
        lat.torch.cuda.synchronize()
        y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc2, Vc2)
        ncp = (nc2 + 7) // 8 * 8
        absl = amg.CoarseLevel(np.abs(level2.A), P2.Lc, nv2)
        rowsum = absl.apply(np.ones(shp2), 0.0).real.reshape(Vc2, nc2)
        for n in range(nsys):
            absb = absl.apply(np.abs(x[n]).reshape(shp2), 0.0).real.reshape(Vc2, nc2)
            absb += abs(mu[n]) * np.abs(x[n])
            xmax = np.abs(np.concatenate([x[n].real.ravel(), x[n].imag.ravel()])).max()
            bound = _f16_bound(absb, rowsum, ncp, xmax) + 1e-6 * np.abs(ref[n])
            err = np.maximum(np.abs(y[n].real - ref[n].real), np.abs(y[n].imag - ref[n].imag))
            assert np.all(err <= bound), (n, (err / bound).max())
    finally:
        lat.close()


def test_middle_and_bottom_coarse_solves():
    # level 1 by the middle FGMRES (level-2 correction + MR smoothing) and level 2 by the bottom
    # solver, each to a tight tolerance, checked with the oracle's level operators
    L, agg, nv, agg2, nv2 = (8, 8, 8, 8), (2, 2, 2, 2), 6, (2, 2, 2, 2), 8
    lat, level1, P2, level2 = _setup3(L, agg, nv, agg2, nv2)
    T = lat.T
    try:
        nrhs, mus = 2, [0.01, 0.2]
        nsys = nrhs * len(mus)
        sp = T.solve_params(mid_tol=1e-5, mid_restart=20, mid_maxiter=200, coarse_tol=1e-5, coarse_restart=30,
                            coarse_maxiter=600, coarse_precision=32)
        for lvl, level, Lc, nvl in ((1, level1, level1.L, nv), (2, level2, P2.Lc, nv2)):
            Vc, nc = int(np.prod(Lc)), 2 * nvl
            shp = synth.lattice_shape(Lc) + (2, nvl)
            r = synth.complex_normal(96 + lvl, 1, (nrhs, Vc, nc))
            rs = np.repeat(r, len(mus), axis=0)  # system n = rhs (n / nshift), shift (n % nshift)
            rb = lat.torch.from_numpy(coarse_to_bundle(rs, nc, Vc)).cuda()
            xb = lat.coarse_buffer(nsys, level=lvl)
            it = T.tmamg_coarse_solve(lat.ctx, lvl, rb, xb, nrhs, mus, len(mus), sp)
            lat.torch.cuda.synchronize()
            x = coarse_from_bundle(xb.cpu().numpy(), nsys, nc, Vc)
            for n in range(nsys):
                mu = mus[n % len(mus)]
                res = np.linalg.norm(rs[n] - level.apply(x[n].reshape(shp), mu).reshape(Vc, nc)) / np.linalg.norm(rs[n])
                assert res < 5e-5, (lvl, n, res, it)
    finally:
        lat.close()


def _solve3(L, U, kappa, b, mus, sp_kw, solve_kw):
    lat = Lattice(L, U, kappa, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(levels=3, **sp_kw))
        nrhs = b.shape[0]
        x = np.zeros((nrhs, len(mus)) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve(lat.ctx, b, nrhs, mus, len(mus), x, 0, T.solve_params(**solve_kw))
        return rc, stats, x
    finally:
        lat.close()


@pytest.mark.parametrize("L,agg,nv,agg2,nv2,coarse_solver", [((8, 8, 8, 8), (2, 2, 2, 2), 8, (2, 2, 2, 2), 8, 0),
                                                              ((12, 8, 8, 8), (2, 2, 2, 2), 6, (2, 2, 2, 2), 10, 0),
                                                              ((8, 8, 8, 8), (2, 2, 2, 2), 8, (2, 2, 2, 2), 8, 1)])
def test_three_level_solve(L, agg, nv, agg2, nv2, coarse_solver):
    U = synth.gauge_field(L, 0.3, seed=7)
    kappa = 0.126
    b = synth.gaussian_spinors(L, 2, seed=8)
    mus = [0.001, 0.05]
    rc, stats, x = _solve3(L, U, kappa, b, mus,
                           dict(agg=agg, nv=nv, agg2=agg2, nv2=nv2, sap_block=(2, 2, 2, 2), setup_iters=4),
                           dict(restart=10, tol=1e-10, coarse_solver=coarse_solver))
    op = dirac.Operator(U, kappa, 1.0)
    assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
    for r in range(2):
        for k, mu in enumerate(mus):
            res = np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r])
            assert res <= 1e-10, (r, k, res)
            s = stats[r * len(mus) + k]
            assert s.status == 0 and abs(s.true_rel_res - res) < 1e-11


def test_three_level_argument_checks():
    L = (8, 8, 8, 8)
    U = synth.gauge_field(L, 0.3, seed=7)
    lat = Lattice(L, U, 0.126, 1.0)
    T = lat.T
    try:
        # level-2 aggregate that does not divide the 4^4 level-1 lattice
        with pytest.raises(T.TmamgError):
            T.tmamg_setup(lat.ctx, T.setup_params(levels=3, agg=(2, 2, 2, 2), nv=6, agg2=(3, 2, 2, 2), nv2=8,
                                                  sap_block=(2, 2, 2, 2), setup_iters=0))
        with pytest.raises(T.TmamgError):
            T.tmamg_setup(lat.ctx, T.setup_params(levels=4, agg=(2, 2, 2, 2), nv=6, sap_block=(2, 2, 2, 2)))
        T.tmamg_setup(lat.ctx, T.setup_params(levels=3, agg=(2, 2, 2, 2), nv=6, agg2=(2, 2, 2, 2), nv2=8,
                                              sap_block=(2, 2, 2, 2), setup_iters=1))
        b = synth.gaussian_spinors(L, 1, seed=9)
        x = np.zeros((1, 1) + b.shape[1:], dtype=np.complex128)
        # the FP64 comparator takes two levels only
        with pytest.raises(T.TmamgError):
            T.tmamg_solve(lat.ctx, b, 1, [0.01], 1, x, 0, T.solve_params(precision=64))
        with pytest.raises(T.TmamgError):
            T.tmamg_solve(lat.ctx, b, 1, [0.01], 1, x, 0, T.solve_params(mid_restart=0))
    finally:
        lat.close()

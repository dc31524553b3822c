"""GPU parity of the multigrid components (SAP, P^+, P, D_c) against the FP64 oracle, and
end-to-end solves checked by the oracle's own operator.

Tolerances: components run in FP32 with FP64 reductions where it matters; a relative
error of 2e-5 allows for FP32 rounding through a few MR steps / Gram-Schmidt passes
(unit roundoff 6e-8 times the step count and the condition of the small dots)."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac, sap
from tests.gpu_util import Lattice, coarse_from_bundle, coarse_to_bundle, from_dev, relerr, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.mark.parametrize("L,bs", [((8, 4, 4, 8), (4, 2, 2, 4)), ((8, 8, 8, 8), (4, 4, 4, 4)),
                                  ((4, 4, 4, 4), (2, 2, 2, 2)),
                                  # 256-site blocks take the face-by-face update: one block along x
                                  # (no x faces), and an 8 x 4 x 4 x 2 block (faces of 32 to 128 sites)
                                  ((4, 8, 8, 8), (4, 4, 4, 4)), ((16, 8, 8, 8), (8, 4, 4, 2))])
def test_sap_matches_oracle(L, bs):
    U = synth.gauge_field(L, 0.3, seed=51)
    kappa, c_sw = 0.124, 1.0
    lat = Lattice(L, U, kappa, c_sw)
    try:
        nsys = 3
        r = synth.gaussian_spinors(L, nsys, seed=52)
        mu = np.array([0.001, 0.05, -0.2])
        rb = lat.fine_bundle(r)
        eb = rb.clone()
        lat.T.tmamg_sap(lat.ctx, rb, eb, nsys, mu, bs, 2, 3)
        e = lat.from_fine_bundle(eb, nsys)
        op = dirac.Operator(U, kappa, c_sw)
        e_ref = sap.sap(op, r, mu, bs, cycles=2, mr_steps=3)
        for n in range(nsys):
            assert relerr(e[n], e_ref[n]) < TOL32, (n, relerr(e[n], e_ref[n]))
    finally:
        lat.close()


def _setup_pair(L, agg, nv, kappa=0.125, seed=61):
    U = synth.gauge_field(L, 0.3, seed=seed)
    lat = Lattice(L, U, kappa, 1.0)
    Vt = synth.gaussian_spinors(L, nv, seed=seed + 1).astype(np.complex64)
    T = lat.T
    p = T.setup_params(agg=agg, nv=nv, sap_block=tuple(2 for _ in range(4)), setup_iters=0)
    T.tmamg_setup_from_vectors(lat.ctx, p, to_dev(Vt))
    op = dirac.Operator(U, kappa, 1.0)
    P = amg.Prolongation(amg.FineLevel.to_chi(Vt.astype(np.complex128)), L, agg)
    A = amg.coarse_operator(amg.FineLevel(op), P)
    return lat, op, P, amg.CoarseLevel(A, P.Lc, nv)


@pytest.mark.parametrize("L,agg,nv", [((4, 4, 4, 4), (2, 2, 2, 2), 8), ((8, 4, 4, 8), (4, 2, 2, 4), 12)])
def test_restrict_prolong_match_oracle(L, agg, nv):
    lat, op, P, cl = _setup_pair(L, agg, nv)
    try:
        nsys = 3
        Vc = int(np.prod(P.Lc))
        nc = 2 * nv
        r = synth.gaussian_spinors(L, nsys, seed=71)
        rb = lat.fine_bundle(r)
        cb = lat.coarse_buffer(nsys)
        lat.T.tmamg_restrict(lat.ctx, 1, rb, cb, nsys)
        lat.torch.cuda.synchronize()
        xc = coarse_from_bundle(cb.cpu().numpy(), nsys, nc, Vc)
        ref = P.restrict(amg.FineLevel.to_chi(r)).reshape(nsys, Vc, nc)
        for n in range(nsys):
            assert relerr(xc[n], ref[n]) < TOL32
        # prolongation of a random coarse vector
        y = synth.complex_normal(72, 1, (nsys, Vc, nc))
        yb = lat.torch.from_numpy(coarse_to_bundle(y, nc, Vc)).cuda()
        fb = lat.fine_bundle(np.zeros((nsys,) + r.shape[1:], dtype=np.complex128))
        lat.T.tmamg_prolong(lat.ctx, 1, yb, fb, nsys)
        e = lat.from_fine_bundle(fb, nsys)
        Lxc, Lyc, Lzc, Ltc = P.Lc
        eref = amg.FineLevel.to_spin(P.prolong(y.reshape(nsys, Ltc, Lzc, Lyc, Lxc, 2, nv)))
        for n in range(nsys):
            assert relerr(e[n], eref[n]) < TOL32
    finally:
        lat.close()


@pytest.mark.parametrize("L,agg,nv", [((4, 4, 4, 4), (2, 2, 2, 2), 8), ((8, 4, 4, 8), (4, 2, 2, 4), 12)])
def test_coarse_operator_matches_oracle(L, agg, nv):
    lat, op, P, cl = _setup_pair(L, agg, nv)
    try:
        nsys = 5
        Vc = int(np.prod(P.Lc))
        nc = 2 * nv
        x = synth.complex_normal(81, 1, (nsys, Vc, nc))
        mu = np.linspace(-0.1, 0.3, nsys)
        xb = lat.torch.from_numpy(coarse_to_bundle(x, nc, Vc)).cuda()
        yb = lat.coarse_buffer(nsys)
        lat.T.tmamg_coarse_apply(lat.ctx, 1, xb, yb, nsys, mu, 32)
        lat.torch.cuda.synchronize()
        y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc, Vc)
        Lxc, Lyc, Lzc, Ltc = P.Lc
        ref = cl.apply(x.reshape(nsys, Ltc, Lzc, Lyc, Lxc, 2, nv), mu).reshape(nsys, Vc, nc)
        for n in range(nsys):
            assert relerr(y[n], ref[n]) < TOL32, relerr(y[n], ref[n])
    finally:
        lat.close()


# FP16 tensor-core stencil: both operands are rounded to FP16 (unit roundoff 2^-11 each) and the
# 18 ncp products of one output entry are summed in FP32 (allowing a truncating accumulator,
# 2^-23 per addition); the elementwise bound is therefore (2^-10 + 18 ncp 2^-22) (|A| |x|)_i,
# with (|A| |x|)_i from the oracle's blocks. The power-of-two scaling keeps max |x_n| in
# [1/2, 1), so entries below 2^-14 max|x_n| meet the subnormal grid (absolute 2^-25 max|x_n|).
def _f16_bound(absb, rowsum, ncp, xmax):
    return (2.0 ** -10 + 18 * ncp * 2.0 ** -22) * absb + 2.0 ** -24 * xmax * rowsum


@pytest.mark.parametrize("L,agg,nv,nsys", [((4, 4, 4, 4), (2, 2, 2, 2), 8, 5),
                                           ((8, 4, 4, 8), (4, 2, 2, 4), 12, 21),
                                           ((8, 4, 4, 8), (4, 2, 2, 4), 12, 2)])
def test_coarse_apply_tensor_cores_within_fp16_bound(L, agg, nv, nsys):
    lat, op, P, cl = _setup_pair(L, agg, nv)
    try:
        Vc = int(np.prod(P.Lc))
        nc = 2 * nv
        ncp = (nc + 7) // 8 * 8
        x = synth.complex_normal(82, 1, (nsys, Vc, nc))
        # one zero system and systems far from unit range exercise the per-system scaling
        x[0] = 0
        if nsys > 2:
            x[1] *= 1e-6
            x[2] *= 3e4
        mu = np.linspace(-0.1, 0.3, nsys)
        xb = lat.torch.from_numpy(coarse_to_bundle(x, nc, Vc)).cuda()
        yb = lat.coarse_buffer(nsys)
        lat.T.tmamg_coarse_apply(lat.ctx, 1, xb, yb, nsys, mu, 16)
        lat.torch.cuda.synchronize()
        y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc, Vc)
        Lxc, Lyc, Lzc, Ltc = P.Lc
        shp = (Ltc, Lzc, Lyc, Lxc, 2, nv)
        cl_abs = amg.CoarseLevel(np.abs(cl.A), P.Lc, nv)
        rowsum = cl_abs.apply(np.ones(shp), 0.0).real.reshape(Vc, nc)
        assert np.all(y[0] == 0)
        for n in range(nsys):
            ref = cl.apply(x[n].reshape(shp), mu[n]).reshape(Vc, nc)
            # the twist term stays in FP32 (relative 2^-23 of |mu| |x|)
            absb = cl_abs.apply(np.abs(x[n]).reshape(shp), 0.0).real.reshape(Vc, nc) + abs(mu[n]) * np.abs(x[n])
            bound = _f16_bound(absb, rowsum, ncp, np.abs(x[n]).max())
            err = np.abs(y[n] - ref)
            assert np.all(err <= bound + 1e-300), (n, float((err / np.maximum(bound, 1e-300)).max()))
            if n > 0:
                assert relerr(y[n], ref) < 2e-3
    finally:
        lat.close()


def _solve(L, U, kappa, c_sw, b, mus, sp_kw, solve_kw):
    lat = Lattice(L, U, kappa, c_sw)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(**sp_kw))
        nrhs = b.shape[0]
        x = np.zeros((nrhs, len(mus)) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve(lat.ctx, b, nrhs, mus, len(mus), x, 0, T.solve_params(**solve_kw))
        return rc, stats, x
    finally:
        lat.close()


def test_solve_tiny_configuration():
    # 4^4, eps 0.3, kappa 0.125, c_sw 1, mu 0.01, one Gaussian rhs, 2-level AMG with 2^4
    # aggregates, Nv 8, SAP blocks 2^4, FGMRES(10) to 1e-10
    L = (4, 4, 4, 4)
    U = synth.gauge_field(L, 0.3, seed=1)
    b = synth.gaussian_spinors(L, 1, seed=1, stream=202)
    rc, stats, x = _solve(L, U, 0.125, 1.0, b, [0.01],
                          dict(agg=(2, 2, 2, 2), nv=8, sap_block=(2, 2, 2, 2), setup_iters=3),
                          dict(restart=10, tol=1e-10))
    op = dirac.Operator(U, 0.125, 1.0)
    res = np.linalg.norm(b[0] - op.apply(x[0, 0], 0.01)) / np.linalg.norm(b[0])
    assert rc == 0 and stats[0].status == 0, [(s.status, s.true_rel_res) for s in stats]
    assert res <= 1e-10
    assert abs(stats[0].true_rel_res - res) < 1e-11
    M = op.dense(0.01)
    xd = np.linalg.solve(M, b[0].ravel())
    assert np.linalg.norm(x[0, 0].ravel() - xd) <= np.linalg.cond(M) * 1e-10 * np.linalg.norm(xd)


@pytest.mark.parametrize("coarse_solver,coarse_precision", [(0, 16), (1, 16), (2, 16), (0, 32), (2, 32)])
def test_solve_multi_rhs_multi_shift(coarse_solver, coarse_precision):
    L = (8, 4, 4, 8)
    U = synth.gauge_field(L, 0.3, seed=3)
    kappa = 0.126
    b = synth.gaussian_spinors(L, 3, seed=4)
    mus = [0.001, 0.02, 0.3]
    rc, stats, x = _solve(L, U, kappa, 1.0, b, mus,
                          dict(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4),
                          dict(restart=10, tol=1e-10, coarse_solver=coarse_solver,
                               coarse_precision=coarse_precision))
    op = dirac.Operator(U, kappa, 1.0)
    assert rc == 0
    for r in range(3):
        for k, mu in enumerate(mus):
            res = np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r])
            assert res <= 1e-10, (r, k, res)
            assert stats[r * 3 + k].status == 0


@pytest.mark.parametrize("L,agg,sap_block,nrhs,mus", [((8, 4, 4, 8), (4, 2, 2, 4), (2, 2, 2, 2), 1, [0.01]),
                                                        ((8, 4, 4, 8), (4, 2, 2, 4), (2, 2, 2, 2), 2, [0.001, 0.3]),
                                                        ((8, 8, 8, 8), (4, 4, 4, 4), (4, 4, 4, 4), 1, [0.01])])
def test_solve_plain_fp64(L, agg, sap_block, nrhs, mus):
    # the plain FP64 comparator (precision 64: FGMRES, AMG cycle, SAP, coarse GMRES all in FP64)
    # reaches the same 1e-10 true residual, checked by the oracle operator; the last case uses
    # 4^4 SAP blocks (the block solver's largest shared-memory footprint)
    U = synth.gauge_field(L, 0.3, seed=3)
    kappa = 0.126
    b = synth.gaussian_spinors(L, nrhs, seed=5)
    rc, stats, x = _solve(L, U, kappa, 1.0, b, mus,
                          dict(agg=agg, nv=12, sap_block=sap_block, setup_iters=4),
                          dict(restart=10, tol=1e-10, precision=64))
    op = dirac.Operator(U, kappa, 1.0)
    assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
    for r in range(nrhs):
        for k, mu in enumerate(mus):
            res = np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r])
            assert res <= 1e-10, (r, k, res)
            s = stats[r * len(mus) + k]
            assert s.status == 0 and abs(s.true_rel_res - res) < 1e-11


def test_solve_precision_lattice_persistent_vs_launches():
    # the 16^3 x 32 lattice with 4 point sources: both coarse-solver forms reach 1e-10 and
    # need a similar number of top-level iterations
    L = (16, 16, 16, 32)
    U = synth.gauge_field(L, 0.25, seed=1)
    kappa = 0.1335
    b = synth.point_sources(L)[:4]
    out = {}
    for cs in (0, 2):
        rc, stats, x = _solve(L, U, kappa, 1.0, b, [0.003],
                              dict(agg=(4, 4, 4, 4), nv=24, sap_block=(4, 4, 4, 4), setup_iters=10),
                              dict(restart=20, tol=1e-10, coarse_restart=40, coarse_maxiter=400, coarse_solver=cs))
        assert rc == 0
        assert all(s.status == 0 and s.true_rel_res <= 1e-10 for s in stats)
        out[cs] = stats[0].inner_iters
        if cs == 0:
            op = dirac.Operator(U, kappa, 1.0)
            res = np.linalg.norm(b[1] - op.apply(x[1, 0], 0.003)) / np.linalg.norm(b[1])
            assert res <= 1e-10
    assert abs(out[0] - out[2]) <= max(3, 0.3 * out[2])


def test_inner_fp32_cycles_cut_fp64_refinements():
    # FP32 FGMRES(4) restarted from its FP32 residual inside each FP64 refinement cycle: every system
    # still reaches the FP64 goal (checked by the oracle operator) with fewer FP64 residuals
    L = (8, 4, 4, 8)
    U = synth.gauge_field(L, 0.3, seed=3)
    kappa = 0.126
    b = synth.gaussian_spinors(L, 2, seed=6)
    mus = [0.001, 0.05]
    op = dirac.Operator(U, kappa, 1.0)
    outer = {}
    for ic in (1, 4):
        rc, stats, x = _solve(L, U, kappa, 1.0, b, mus,
                              dict(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4),
                              dict(restart=4, tol=1e-10, inner_cycles=ic))
        assert rc == 0, [(s.status, s.true_rel_res) for s in stats]
        for r in range(2):
            for k, mu in enumerate(mus):
                res = np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r])
                assert res <= 1e-10, (ic, r, k, res)
        outer[ic] = max(s.outer_iters for s in stats)
    assert outer[4] < outer[1], outer


def test_solve_time_sap_settings_override_the_setup():
    # the AMG cycle's SAP takes its cycles and MR steps from the solve parameters when they are set
    # (the setup's smoothing keeps its own): both forms reach 1e-10, the iteration counts differ, and
    # negative values are rejected
    L = (8, 4, 4, 8)
    U = synth.gauge_field(L, 0.3, seed=3)
    kappa = 0.126
    b = synth.gaussian_spinors(L, 2, seed=4)
    mus = [0.001, 0.05]
    lat = Lattice(L, U, kappa, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4,
                                              sap_mr_steps=6))
        its = []
        for kw in (dict(), dict(sap_cycles=1, sap_mr_steps=1)):
            x = np.zeros((2, 2) + b.shape[1:], dtype=np.complex128)
            rc, stats = T.tmamg_solve(lat.ctx, b, 2, mus, 2, x, 0, T.solve_params(restart=10, tol=1e-10, **kw))
            assert rc == 0 and all(s.status == 0 for s in stats)
            op = dirac.Operator(U, kappa, 1.0)
            for r in range(2):
                for k, mu in enumerate(mus):
                    assert np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r]) <= 1e-10
            its.append(max(s.inner_iters for s in stats))
        assert its[1] > its[0], its
        x = np.zeros((2, 2) + b.shape[1:], dtype=np.complex128)
        with pytest.raises(T.TmamgError):
            T.tmamg_solve(lat.ctx, b, 2, mus, 2, x, 0, T.solve_params(sap_mr_steps=-1))
    finally:
        lat.close()

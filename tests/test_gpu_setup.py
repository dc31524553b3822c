"""GPU parity of the multigrid setup's smoothing (paper Sec. 2: test vectors that approximate
low modes by inverse iteration) against the FP64 oracle. The same start vectors are smoothed on
the GPU (tmamg_setup with setup_iters > 0: SAP inverse iteration on the fine level, level-1
GMRES inverse iteration for the second coarse level) and by oracle.amg.setup_test_vectors /
setup_coarse_test_vectors; the prolongations built from the two sets must agree, compared
through restrictions of random vectors.

Tolerance: every smoothing step is an FP32 SAP application (its own parity bar against the
oracle is 2e-5) or FP32 GMRES steps, then a normalisation. Gram-Schmidt on an aggregate's
pieces amplifies a relative perturbation of the vectors by at most the condition number of that
aggregate's vector block (sigma_max / sigma_min), which the test computes from the oracle's
vectors. The bar is iterations x 2e-5 x the largest condition number."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac
from tests.gpu_util import Lattice, coarse_from_bundle, coarse_to_bundle, relerr

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _max_cond(V, L, agg):
    """Largest condition number over aggregates x chiralities of the vector blocks of V [Nv, ..., 2, d]."""
    Va = amg.to_agg(V, L, agg, 2)                       # [Nv, Vc, |a|, 2, d]
    X = Va.transpose(1, 3, 2, 4, 0)                    # [Vc, 2, |a|, d, Nv]
    X = X.reshape(X.shape[0], 2, -1, X.shape[-1])
    s = np.linalg.svd(X, compute_uv=False)
    return float((s[..., 0] / s[..., -1]).max())


@pytest.mark.parametrize("L,agg,nv,sap_block,iters", [((8, 4, 4, 8), (4, 2, 2, 4), 12, (4, 2, 2, 4), 3),
                                                      ((8, 8, 8, 8), (4, 4, 4, 4), 24, (4, 4, 4, 4), 2)])
def test_setup_smoothing_matches_oracle(L, agg, nv, sap_block, iters):
    U = synth.gauge_field(L, 0.3, seed=111)
    kappa, c_sw, mu_setup = 0.125, 1.0, 0.0
    lat = Lattice(L, U, kappa, c_sw)
    try:
        T = lat.T
        V0 = synth.gaussian_spinors(L, nv, seed=112).astype(np.complex64)
        p = T.setup_params(agg=agg, nv=nv, sap_block=sap_block, setup_iters=iters, mu_setup=mu_setup)
        dev = lat.torch.from_numpy(V0.view(np.float32).copy()).cuda()
        T.tmamg_setup(lat.ctx, p, dev)
        op = dirac.Operator(U, kappa, c_sw)
        V = amg.setup_test_vectors(op, V0.astype(np.complex128), mu_setup, sap_block, iters, sap_cycles=2, mr_steps=3)
        Vchi = amg.FineLevel.to_chi(V)
        P = amg.Prolongation(Vchi, L, agg)
        tol = iters * TOL32 * _max_cond(Vchi, L, agg)
        nsys = 4
        Vc, nc = int(np.prod(P.Lc)), 2 * nv
        r = synth.gaussian_spinors(L, nsys, seed=113)
        cb = lat.coarse_buffer(nsys)
        T.tmamg_restrict(lat.ctx, 1, lat.fine_bundle(r), cb, nsys)
        lat.torch.cuda.synchronize()
        got = coarse_from_bundle(cb.cpu().numpy(), nsys, nc, Vc)
        ref = P.restrict(amg.FineLevel.to_chi(r)).reshape(nsys, Vc, nc)
        for n in range(nsys):
            assert relerr(got[n], ref[n]) < tol, (n, relerr(got[n], ref[n]), tol)
    finally:
        lat.close()


def test_level2_setup_smoothing_matches_oracle():
    # three levels: both levels' vectors smoothed (SAP inverse iteration on the fine level, then
    # inverse iteration with 12 steps of level-1 GMRES for the level-2 vectors)
    L, agg, nv, agg2, nv2 = (8, 4, 4, 8), (2, 2, 2, 2), 8, (2, 1, 1, 2), 10
    sap_block, iters, gsteps = (2, 2, 2, 2), 2, 12
    U = synth.gauge_field(L, 0.3, seed=121)
    kappa, c_sw, mu_setup = 0.125, 1.0, 0.0
    lat = Lattice(L, U, kappa, c_sw)
    try:
        T = lat.T
        V0 = synth.gaussian_spinors(L, nv, seed=122).astype(np.complex64)
        Lc1 = amg.coarse_extent(L, agg)
        W0 = synth.gaussian_coarse(Lc1, nv2, nv, seed=123).astype(np.complex64)
        vecs = np.concatenate([V0.ravel(), W0.ravel()])
        p = T.setup_params(levels=3, agg=agg, nv=nv, sap_block=sap_block, setup_iters=iters, mu_setup=mu_setup,
                           agg2=agg2, nv2=nv2, setup_gmres_steps=gsteps)
        T.tmamg_setup(lat.ctx, p, lat.torch.from_numpy(vecs.view(np.float32).copy()).cuda())
        op = dirac.Operator(U, kappa, c_sw)
        three = amg.ThreeLevelAMG(op, agg, V0.astype(np.complex128), sap_block, agg2, W0.astype(np.complex128),
                                  setup_iters=iters, mu_setup=mu_setup, setup_gmres_steps=gsteps)
        tol1 = iters * TOL32 * _max_cond(amg.FineLevel.to_chi(three.two.V), L, agg)
        tol2 = tol1 + iters * TOL32 * _max_cond(three.W, Lc1, agg2)
        nsys = 3
        # level 1: the fine vectors' smoothing
        Vc1, nc1 = int(np.prod(Lc1)), 2 * nv
        r = synth.gaussian_spinors(L, nsys, seed=124)
        cb1 = lat.coarse_buffer(nsys, level=1)
        T.tmamg_restrict(lat.ctx, 1, lat.fine_bundle(r), cb1, nsys)
        lat.torch.cuda.synchronize()
        got1 = coarse_from_bundle(cb1.cpu().numpy(), nsys, nc1, Vc1)
        ref1 = three.P1.restrict(amg.FineLevel.to_chi(r)).reshape(nsys, Vc1, nc1)
        for n in range(nsys):
            assert relerr(got1[n], ref1[n]) < tol1, (n, relerr(got1[n], ref1[n]), tol1)
        # level 2: P2 from the level-1 GMRES smoothing, compared on random level-1 vectors
        Vc2, nc2 = int(np.prod(three.P2.Lc)), 2 * nv2
        x1 = synth.complex_normal(125, 1, (nsys, Vc1, nc1))
        cb2 = lat.coarse_buffer(nsys, level=2)
        T.tmamg_restrict(lat.ctx, 2, lat.torch.from_numpy(coarse_to_bundle(x1, nc1, Vc1)).cuda(), cb2, nsys)
        lat.torch.cuda.synchronize()
        got2 = coarse_from_bundle(cb2.cpu().numpy(), nsys, nc2, Vc2)
        shp1 = synth.lattice_shape(Lc1) + (2, nv)
        ref2 = three.P2.restrict(x1.reshape((nsys,) + shp1)).reshape(nsys, Vc2, nc2)
        for n in range(nsys):
            assert relerr(got2[n], ref2[n]) < tol2, (n, relerr(got2[n], ref2[n]), tol2)
    finally:
        lat.close()

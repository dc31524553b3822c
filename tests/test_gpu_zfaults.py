"""Failure behaviour of the solver on the GPU without any device fault: a right-hand side with a NaN
is reported as non-finite for its own system only (the other systems still reach 1e-10), and a
refinement cap below what the goal needs returns TMAMG_NOT_CONVERGED with every system's statistics
written. Both failures are made on the host (the input, the parameters)."""
import numpy as np
import pytest

import synth
from oracle import dirac
from tests.gpu_util import Lattice

pytestmark = pytest.mark.gpu

L = (8, 4, 4, 8)
KAPPA = 0.126


def _lattice():
    U = synth.gauge_field(L, 0.3, seed=3)
    lat = Lattice(L, U, KAPPA, 1.0)
    T = lat.T
    T.tmamg_setup(lat.ctx, T.setup_params(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=3))
    return U, lat


def test_nan_rhs_is_reported_for_its_system_only():
    U, lat = _lattice()
    T = lat.T
    try:
        b = synth.gaussian_spinors(L, 3, seed=41)
        b[1, 0, 0, 0, 0, 0, 0] = np.nan
        x = np.zeros((3, 1) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve(lat.ctx, b, 3, [0.01], 1, x, 0, T.solve_params())
        assert rc == T.TMAMG_NOT_CONVERGED
        assert stats[1].status == -5  # TMAMG_ERR_NONFINITE
        op = dirac.Operator(U, KAPPA, 1.0)
        for r in (0, 2):
            assert stats[r].status == 0
            res = np.linalg.norm(b[r] - op.apply(x[r, 0], 0.01)) / np.linalg.norm(b[r])
            assert res <= 1e-10, (r, res)
    finally:
        lat.close()


def test_refinement_cap_returns_not_converged_with_stats():
    U, lat = _lattice()
    T = lat.T
    try:
        b = synth.gaussian_spinors(L, 2, seed=42)
        mus = [0.001, 0.1]
        x = np.zeros((2, 2) + b.shape[1:], dtype=np.complex128)
        # one refinement cycle of FGMRES(2) cannot reach 1e-14
        rc, stats = T.tmamg_solve(lat.ctx, b, 2, mus, 2, x, 0, T.solve_params(tol=1e-14, max_outer=1, restart=2))
        assert rc == T.TMAMG_NOT_CONVERGED
        op = dirac.Operator(U, KAPPA, 1.0)
        for r in range(2):
            for k, mu in enumerate(mus):
                s = stats[r * 2 + k]
                assert s.status == T.TMAMG_NOT_CONVERGED and s.outer_iters == 1 and s.inner_iters >= 1
                res = np.linalg.norm(b[r] - op.apply(x[r, k], mu)) / np.linalg.norm(b[r])
                # x is the partial solution and the reported residual is its true residual
                assert 1e-14 < res < 1.0 and abs(s.true_rel_res - res) <= 1e-3 * res, (r, k, res, s.true_rel_res)
    finally:
        lat.close()


def test_coarse_barrier_timeout_is_reported_and_context_recovers():
    # the persistent coarse GMRES's grid barrier is made unreachable from the host (it waits for one
    # arrival more than the grid holds) with a 10 ms bound; the first barrier follows a plain vector
    # pass and the FP32 stencil is used, so no bulk copy or tensor-core work is in flight when the
    # wait gives up. The call must report TMAMG_ERR_TIMEOUT and the context must still solve.
    U, lat = _lattice()
    T = lat.T
    try:
        nrhs, mus = 2, [0.01]
        nsys = nrhs * len(mus)
        nc = 24
        Vc = int(np.prod([8 // 4, 4 // 2, 4 // 2, 8 // 4]))
        from tests.gpu_util import coarse_to_bundle
        rc_vec = synth.complex_normal(43, 1, (nsys, Vc, nc))
        rb = lat.torch.from_numpy(coarse_to_bundle(rc_vec, nc, Vc)).cuda()
        xb = lat.coarse_buffer(nsys)
        sp = T.solve_params(coarse_precision=32, coarse_solver=0, coarse_tol=1e-3, coarse_maxiter=200)
        T.tmamg_debug_bounded_wait(20_000_000, 1)  # about 10 ms at 2 GHz
        try:
            with pytest.raises(T.TmamgError) as ei:
                T.tmamg_coarse_solve(lat.ctx, 1, rb, xb, nrhs, mus, len(mus), sp)
            assert ei.value.code == -6, ei.value  # TMAMG_ERR_TIMEOUT
        finally:
            T.tmamg_debug_bounded_wait(0, 0)
        # the same call without the unreachable barrier converges
        it = T.tmamg_coarse_solve(lat.ctx, 1, rb, xb, nrhs, mus, len(mus), sp)
        assert 0 < it < 200
        yb = lat.coarse_buffer(nsys)
        T.tmamg_coarse_apply(lat.ctx, 1, xb, yb, nsys, np.array(mus * nrhs), 32)
        lat.torch.cuda.synchronize()
        from tests.gpu_util import coarse_from_bundle
        y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc, Vc)
        for n in range(nsys):
            assert np.linalg.norm(y[n] - rc_vec[n]) <= 2e-3 * np.linalg.norm(rc_vec[n]), n
    finally:
        lat.close()

"""GPU parity at the shapes the benchmark runs, against the FP64 oracle.

* the fine stencil on the 16^3 x 32 lattice with 12 distinct systems (6 tiles of two, the
  benchmark's CTA shape of 32 sites x 6 tiles), every system compared;
* restriction and prolongation with 4^4 aggregates and Nv = 24 (256-site aggregates, the
  staging-chunk path of the benchmark);
* the coarse stencil with 4^4 aggregates at Nv = 24 (n_c = 48, the first coarse level of the
  benchmark) and Nv = 32 (n_c = 64, the second coarse level of the three-level hierarchy), in FP32
  and on the tensor cores in FP16, for 12 and 16 systems.

Tolerances as in the component tests: FP32 components 2e-5 relative (the fine stencil 1e-6,
the FP32 operator bar), the FP16 stencil elementwise within the rounding bound of its two FP16
operands and FP32 sums."""
import numpy as np
import pytest

import synth
from oracle import amg, dirac
from tests.gpu_util import coarse_from_bundle, coarse_to_bundle, from_dev, relerr, to_dev, torch_cuda
from tests.test_gpu_amg import _f16_bound, _setup_pair

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def test_dirac_precision_lattice_twelve_distinct_systems():
    torch = torch_cuda()
    from paper_2201_03872_gb300 import tmamg as T
    L = (16, 16, 16, 32)
    U = synth.gauge_field(L, 0.25, seed=1)
    kappa = 0.1294
    ctx = T.tmamg_create(L, -1)
    try:
        T.tmamg_load_gauge(ctx, U)
        T.tmamg_set_operator(ctx, kappa, 1.0)
        nsys = 12
        x = synth.gaussian_spinors(L, nsys, seed=45)
        mu = np.linspace(-0.01, 0.05, nsys)  # a different twisted mass in every lane and tile
        xd = to_dev(x.astype(np.complex64))
        yd = torch.empty_like(xd)
        nb = T.tmamg_bundle_bytes(ctx, nsys, 32)
        xb = torch.empty(nb // 4, dtype=torch.float32, device="cuda")
        yb = torch.empty_like(xb)
        T.tmamg_pack(ctx, xd, xb, nsys, 32)
        T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32)
        T.tmamg_unpack(ctx, yb, yd, nsys, 32)
        y = from_dev(yd, x.shape, np.complex64).astype(np.complex128)
        y_ref = dirac.Operator(U, kappa, 1.0).apply(x.astype(np.complex64).astype(np.complex128), mu)
        for n in range(nsys):
            assert relerr(y[n], y_ref[n]) <= 1e-6, (n, relerr(y[n], y_ref[n]))
            assert np.abs(y[n] - y_ref[n]).max() <= 2e-6 * np.abs(y_ref[n]).max(), n
    finally:
        T.tmamg_destroy(ctx)


def test_restrict_prolong_bench_shape():
    L, agg, nv = (8, 8, 8, 8), (4, 4, 4, 4), 24
    lat, op, P, cl = _setup_pair(L, agg, nv)
    try:
        nsys = 12
        Vc, nc = int(np.prod(P.Lc)), 2 * nv
        r = synth.gaussian_spinors(L, nsys, seed=131)
        cb = lat.coarse_buffer(nsys)
        lat.T.tmamg_restrict(lat.ctx, 1, lat.fine_bundle(r), cb, nsys)
        lat.torch.cuda.synchronize()
        xc = coarse_from_bundle(cb.cpu().numpy(), nsys, nc, Vc)
        ref = P.restrict(amg.FineLevel.to_chi(r)).reshape(nsys, Vc, nc)
        for n in range(nsys):
            assert relerr(xc[n], ref[n]) < TOL32, (n, relerr(xc[n], ref[n]))
        y = synth.complex_normal(132, 1, (nsys, Vc, nc))
        yb = lat.torch.from_numpy(coarse_to_bundle(y, nc, Vc)).cuda()
        fb = lat.fine_bundle(np.zeros((nsys,) + r.shape[1:], dtype=np.complex128))
        lat.T.tmamg_prolong(lat.ctx, 1, yb, fb, nsys)
        e = lat.from_fine_bundle(fb, nsys)
        eref = amg.FineLevel.to_spin(P.prolong(y.reshape((nsys,) + synth.lattice_shape(P.Lc) + (2, nv))))
        for n in range(nsys):
            assert relerr(e[n], eref[n]) < TOL32, (n, relerr(e[n], eref[n]))
    finally:
        lat.close()


@pytest.mark.parametrize("nv,nsys", [(24, 12), (24, 16), (32, 16), (32, 12)])
def test_coarse_apply_bench_shapes(nv, nsys):
    L, agg = (8, 8, 8, 8), (4, 4, 4, 4)
    lat, op, P, cl = _setup_pair(L, agg, nv)
    try:
        Vc, nc = int(np.prod(P.Lc)), 2 * nv
        ncp = (nc + 7) // 8 * 8
        shp = synth.lattice_shape(P.Lc) + (2, nv)
        x = synth.complex_normal(133, 1, (nsys, Vc, nc))
        x[1] *= 1e-5  # per-system scaling far from unit range
        mu = np.linspace(-0.05, 0.2, nsys)
        xb = lat.torch.from_numpy(coarse_to_bundle(x, nc, Vc)).cuda()
        cl_abs = amg.CoarseLevel(np.abs(cl.A), P.Lc, nv)
        rowsum = cl_abs.apply(np.ones(shp), 0.0).real.reshape(Vc, nc)
        for prec in (32, 16):
            yb = lat.coarse_buffer(nsys)
            lat.T.tmamg_coarse_apply(lat.ctx, 1, xb, yb, nsys, mu, prec)
            lat.torch.cuda.synchronize()
            y = coarse_from_bundle(yb.cpu().numpy(), nsys, nc, Vc)
            for n in range(nsys):
                ref = cl.apply(x[n].reshape(shp), mu[n]).reshape(Vc, nc)
                if prec == 32:
                    assert relerr(y[n], ref) < TOL32, (n, relerr(y[n], ref))
                    continue
                absb = cl_abs.apply(np.abs(x[n]).reshape(shp), 0.0).real.reshape(Vc, nc) + abs(mu[n]) * np.abs(x[n])
                bound = _f16_bound(absb, rowsum, ncp, np.abs(x[n]).max())
                err = np.abs(y[n] - ref)
                assert np.all(err <= bound + 1e-300), (n, float((err / np.maximum(bound, 1e-300)).max()))
    finally:
        lat.close()

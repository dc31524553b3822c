"""The allocation-free SAP entry point (tmamg_sap_noalloc) gives the same result as tmamg_sap.

It exists for callers that cannot allocate device memory at call time, such as code running
during CUDA stream capture or under a memory budget fixed in advance. This file is collected
last so that a run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import numpy as np
import pytest

import synth
from tests.gpu_util import Lattice, relerr

pytestmark = pytest.mark.gpu

TOL32 = 2e-5  # the tolerance of the other FP32 SAP parity tests


def test_sap_noalloc_matches_sap_twice():
    L = (8, 4, 4, 8)
    bs = (4, 2, 2, 4)
    U = synth.gauge_field(L, 0.3, seed=91)
    lat = Lattice(L, U, 0.124, 1.0)
    try:
        T = lat.T
        nsys = 3
        mu = np.array([0.002, -0.05, 0.3])
        r = synth.gaussian_spinors(L, nsys, seed=92)
        rb = lat.fine_bundle(r)
        eb = lat.torch.zeros_like(rb)
        T.tmamg_sap(lat.ctx, rb, eb, nsys, mu, bs, 2, 3)
        e_ref = lat.from_fine_bundle(eb, nsys)
        r_ref = lat.from_fine_bundle(rb, nsys)  # both calls leave the partially updated residual in r
        for call in range(2):
            rb2 = lat.fine_bundle(r)
            eb2 = lat.torch.full_like(rb2, 7.0)  # the output need not be cleared by the caller
            T.tmamg_sap_noalloc(lat.ctx, rb2, eb2, nsys, mu, bs, 2, 3)
            lat.torch.cuda.synchronize()  # the call returns without waiting for its stream
            e = lat.from_fine_bundle(eb2, nsys)
            r2 = lat.from_fine_bundle(rb2, nsys)
            for n in range(nsys):
                assert relerr(e[n], e_ref[n]) <= TOL32, (call, n, relerr(e[n], e_ref[n]))
                assert relerr(r2[n], r_ref[n]) <= TOL32, (call, n, relerr(r2[n], r_ref[n]))
    finally:
        lat.close()


def test_sap_noalloc_rejects_oversized_bundle():
    from paper_2201_03872_gb300 import tmamg as T
    L = (16, 16, 16, 32)
    lat = Lattice(L, synth.unit_gauge(L), 0.12, 1.0)
    try:
        nsys = 8  # 4 tiles x 12 x 131072 sites x 16 bytes = 100 MB > 64 MiB of scratch
        rb = lat.torch.zeros(T.tmamg_bundle_bytes(lat.ctx, nsys, 32) // 4, dtype=lat.torch.float32, device="cuda")
        eb = lat.torch.zeros_like(rb)
        with pytest.raises(T.TmamgError) as ei:
            T.tmamg_sap_noalloc(lat.ctx, rb, eb, nsys, np.zeros(nsys), (4, 4, 4, 4), 1, 1)
        assert ei.value.code == -1 and "scratch" in str(ei.value)
    finally:
        lat.close()


def test_sap_noalloc_rejects_too_many_systems():
    from paper_2201_03872_gb300 import tmamg as T
    L = (4, 4, 4, 4)
    lat = Lattice(L, synth.unit_gauge(L), 0.12, 1.0)
    try:
        nsys = 65  # one more than the fixed twisted-mass array holds; 33 tiles of this lattice fit the scratch
        rb = lat.torch.zeros(T.tmamg_bundle_bytes(lat.ctx, nsys, 32) // 4, dtype=lat.torch.float32, device="cuda")
        eb = lat.torch.zeros_like(rb)
        with pytest.raises(T.TmamgError) as ei:
            T.tmamg_sap_noalloc(lat.ctx, rb, eb, nsys, np.zeros(nsys), (2, 2, 2, 2), 1, 1)
        assert ei.value.code == -1 and "systems" in str(ei.value)
    finally:
        lat.close()

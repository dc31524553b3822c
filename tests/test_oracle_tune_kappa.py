"""Pin for the kappa-tuning helper of the workload preparation: on the free field (all links 1,
where the clover term vanishes) the singular values of D_W are known in closed form, one per lattice
momentum: sigma(p)^2 = (1/(2 kappa) - sum_mu cos p_mu)^2 + sum_mu sin^2 p_mu, with periodic momenta
in x, y, z and antiperiodic ones in t. Lanczos through the oracle operator must find both ends."""
import numpy as np
import pytest

import synth
from oracle import dirac
from oracle.tune_kappa import singular_extremes


def _closed_form(L, kappa):
    Lx, Ly, Lz, Lt = L
    px = 2 * np.pi * np.arange(Lx) / Lx
    py = 2 * np.pi * np.arange(Ly) / Ly
    pz = 2 * np.pi * np.arange(Lz) / Lz
    pt = (2 * np.arange(Lt) + 1) * np.pi / Lt
    P = np.meshgrid(px, py, pz, pt, indexing="ij")
    a = 1.0 / (2 * kappa) - sum(np.cos(p) for p in P)
    b = sum(np.sin(p) ** 2 for p in P)
    s = np.sqrt(a ** 2 + b)
    return s.min(), s.max()


@pytest.mark.parametrize("kappa", [0.125, 0.11])
def test_free_field_singular_extremes(kappa):
    L = (4, 4, 4, 4)
    op = dirac.Operator(synth.unit_gauge(L), kappa, 1.0, bc_t=-1)
    smin, smax = singular_extremes(op, tol=1e-8)
    ref_min, ref_max = _closed_form(L, kappa)
    assert abs(smin - ref_min) < 1e-5 * ref_max
    assert abs(smax - ref_max) < 2e-3 * ref_max  # the largest end is taken with eigsh tol 1e-3

"""Pins for the seeded input generators (workload prep shared by oracle and CUDA path)."""
import numpy as np

import synth
from oracle.dirac import plaquette


def test_splitmix64_published_sequence():
    # splitmix64 from state 0 (Steele, Lea, Flood 2014): its first four outputs
    z = synth._splitmix64(np.arange(4, dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                   0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_normal_moments():
    z = synth.normal(7, 1, 200000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01


def test_gauge_field_is_su3():
    U = synth.gauge_field((4, 4, 2, 4), 0.3, seed=3)
    I = np.einsum("...ab,...cb->...ac", U, U.conj())
    assert np.abs(I - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


def test_plaquette_small_eps():
    # U = exp(i eps H): 1 - <plaq> shrinks like eps^2
    L = (4, 4, 4, 4)
    p1 = 1 - plaquette(synth.gauge_field(L, 0.05, seed=1))
    p2 = 1 - plaquette(synth.gauge_field(L, 0.1, seed=1))
    assert 0 < p1 < p2
    assert 3.0 < p2 / p1 < 5.0
    assert abs(plaquette(synth.unit_gauge(L)) - 1.0) < 1e-15


def test_z2_noise_and_point_sources():
    z = synth.z2_spinors((2, 2, 2, 2), 3, seed=1)
    assert np.allclose(np.abs(z), 1.0)
    assert np.allclose(np.abs(z.real), 1 / np.sqrt(2))
    b = synth.point_sources((2, 2, 2, 4))
    assert b.shape == (12, 4, 2, 2, 2, 4, 3)
    assert np.allclose(b.reshape(12, -1).sum(axis=1), 1.0)
    mus = synth.log_shifts(10)
    assert np.isclose(mus[0], 1e-3) and np.isclose(mus[-1], 1e-1)


def test_split_generation_gives_the_same_numbers():
    # large inputs are generated in chunks (threads for Gaussian vectors, spawned processes for
    # links); every split must reproduce the whole-array recipe exactly
    import numpy as np
    n = (1 << 20) + 777
    z = synth.normal(5, 9, 2 * n) * np.sqrt(0.5)
    assert np.array_equal(synth.complex_normal(5, 9, (n,)), z[:n] + 1j * z[n:])
    L = (4, 4, 4, 8)
    whole = synth.gauge_field(L, 0.3, seed=2, chunk=1 << 20, processes=1)
    split = synth.gauge_field(L, 0.3, seed=2, chunk=500, processes=2)
    assert np.array_equal(whole, split)

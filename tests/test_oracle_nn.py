"""Pins for the oracle parallel-transport network: identity weights, transport adjoints,
gauge equivariance and finite-difference gradients (FP64)."""
import numpy as np
import pytest

import synth
from oracle import dirac, nn

L = (4, 2, 2, 4)


@pytest.fixture(scope="module")
def tr():
    return nn.Transport(synth.gauge_field(L, 0.4, seed=201), bc_t=-1)


def _field(ch, seed, batch=2):
    return synth.complex_normal(seed, 1, (batch, L[3], L[2], L[1], L[0], ch, 3))


def test_identity_weights(tr):
    Ws = nn.init_weights(identity=True, scale=0.0)
    r = _field(4, 202)
    y, _ = nn.forward(tr, Ws, r)
    assert np.abs(y - r).max() < 1e-15


@pytest.mark.parametrize("h", range(9))
def test_transport_adjoint(tr, h):
    x, y = _field(3, 203, 1), _field(3, 204, 1)
    lhs = np.vdot(y, tr.apply(x, h))
    rhs = np.vdot(tr.adjoint(y, h), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_transport_is_the_hop_of_the_operator(tr):
    # the forward hop of D is -1/2 (1 - gamma_nu) T_{+nu}: check T against the operator's hop
    op = dirac.Operator(tr.U, 0.12, 0.0)
    x = _field(4, 205, 1)[0]
    for nu in range(4):
        ref = op.hop_fwd(x, nu)
        mine = -0.5 * np.einsum("st,...tc->...sc", op.eye4 - op.g[nu], tr.apply(x, 1 + 2 * nu))
        assert np.abs(ref - mine).max() < 1e-14


def test_gauge_equivariance(tr):
    V = int(np.prod(L))
    G = synth.random_su3(V, seed=206).reshape((L[3], L[2], L[1], L[0], 3, 3))
    U = tr.U
    Up = np.empty_like(U)
    for nu in range(4):
        disp = [1 if d == nu else 0 for d in range(4)]
        Up[..., nu, :, :] = G @ U[..., nu, :, :] @ dirac.dag(dirac.link_shift(G, disp))
    trp = nn.Transport(Up, bc_t=-1)
    Ws = nn.init_weights(seed=3, scale=1.0, identity=False)
    r = _field(4, 207)
    Gr = np.einsum("...ab,n...kb->n...ka", G, r)
    lhs, _ = nn.forward(trp, Ws, Gr)
    y, _ = nn.forward(tr, Ws, r)
    rhs = np.einsum("...ab,n...kb->n...ka", G, y)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_finite_difference_gradient(tr):
    Ws = nn.init_weights(seed=5, scale=1.0, identity=True)
    r, e = _field(4, 208), _field(4, 209)
    loss, grads = nn.loss_and_grad(tr, Ws, r, e)
    rng_idx = synth.uniform(9, 1, 24)
    eps = 1e-6
    for k in range(12):
        l = int(rng_idx[k] * 3) % 3
        W = Ws[l]
        flat = int(rng_idx[k + 12] * W.size) % W.size
        for direction in (1.0, 1j):
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[l].flat[flat] += eps * direction
            Wm[l].flat[flat] -= eps * direction
            fd = (nn.loss_and_grad(tr, Wp, r, e)[0] - nn.loss_and_grad(tr, Wm, r, e)[0]) / (2 * eps)
            an = (np.conj(grads[l].flat[flat]) * direction).real
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (l, flat, direction, fd, an)

"""GPU kernels of the learned preconditioner step against the FP64 oracle network:
forward (FP32 weights <= 1e-5; BF16 inference weights within their rounding), loss and
weight gradients (<= 1e-4), and a small training run with the gate (plain SAP judges)."""
import numpy as np
import pytest

import synth
from oracle import nn as onn
from tests.gpu_util import Lattice, relerr

pytestmark = pytest.mark.gpu

L = (8, 4, 4, 8)


@pytest.fixture(scope="module")
def setup():
    U = synth.gauge_field(L, 0.3, seed=301)
    lat = Lattice(L, U, 0.125, 1.0)
    tr = onn.Transport(U, bc_t=-1)
    Ws = onn.init_weights(seed=11, scale=1.0, identity=True)
    lat.T.tmamg_nn_set_weights(lat.ctx, Ws)
    yield lat, tr, Ws
    lat.close()


def test_forward_matches_oracle(setup):
    lat, tr, Ws = setup
    nsys = 3
    r = synth.gaussian_spinors(L, nsys, seed=302)
    rb = lat.fine_bundle(r)
    yb = lat.torch.zeros_like(rb)
    lat.T.tmamg_nn_forward(lat.ctx, rb, yb, nsys, bf16=False)
    y = lat.from_fine_bundle(yb, nsys)
    ref, _ = onn.forward(tr, Ws, r.reshape(r.shape[:-2] + (4, 3)))
    for n in range(nsys):
        assert relerr(y[n], ref[n]) < 1e-5, relerr(y[n], ref[n])
    # BF16 inference weights: the error is the weights' rounding (2^-8 relative), not more
    lat.T.tmamg_nn_forward(lat.ctx, rb, yb, nsys, bf16=True)
    yh = lat.from_fine_bundle(yb, nsys)
    for n in range(nsys):
        assert relerr(yh[n], ref[n]) < 2e-2


def test_loss_and_gradient_match_oracle(setup):
    lat, tr, Ws = setup
    nsys = 3
    r = synth.gaussian_spinors(L, nsys, seed=303)
    e = synth.gaussian_spinors(L, nsys, seed=304)
    loss, grad = lat.T.tmamg_nn_loss_grad(lat.ctx, lat.fine_bundle(r), lat.fine_bundle(e), nsys)
    rl, gl = onn.loss_and_grad(tr, Ws, r.astype(np.complex64).astype(np.complex128),
                               e.astype(np.complex64).astype(np.complex128))
    assert abs(loss - rl) < 1e-5 * rl
    ref = np.concatenate([g.ravel() for g in gl])
    assert relerr(grad, ref) < 1e-4, relerr(grad, ref)


def test_training_lowers_loss_and_gate_is_consistent():
    U = synth.gauge_field(L, 0.3, seed=305)
    lat = Lattice(L, U, 0.126, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4))
        rep = T.tmamg_nn_train(lat.ctx, T.tmamg_default_nn_params(pairs=24, batch=6, epochs=20, lr=3e-3, mu=0.001,
                                                                 gate_systems=4))
        assert rep.loss_last < rep.loss_first, (rep.loss_first, rep.loss_last)
        assert rep.enabled == (1 if rep.iters_nn < rep.iters_plain else 0)
        # with the step forced on, FGMRES still reaches the FP64 goal
        b = synth.gaussian_spinors(L, 2, seed=306)
        x = np.zeros((2, 1) + b.shape[1:], dtype=np.complex128)
        rc, stats = T.tmamg_solve(lat.ctx, b, 2, [0.001], 1, x, 0, T.solve_params(use_nn=2))
        assert rc == 0 and all(s.true_rel_res <= 1e-10 for s in stats)
        print(f"nn gate: plain {rep.iters_plain} iterations, with the learned step {rep.iters_nn}, "
              f"loss {rep.loss_first:.3f} -> {rep.loss_last:.3f}, enabled {rep.enabled}")
    finally:
        lat.close()


def test_windowed_training_matches_single_window_and_lowers_loss():
    # pairs collected and trained window by window (4 batches resident at a time over 12 batches):
    # the loss falls, and with one window covering every batch the windowed form is the plain one
    U = synth.gauge_field(L, 0.3, seed=307)
    lat = Lattice(L, U, 0.126, 1.0)
    T = lat.T
    try:
        T.tmamg_setup(lat.ctx, T.setup_params(agg=(4, 2, 2, 4), nv=12, sap_block=(2, 2, 2, 2), setup_iters=4))
        kw = dict(pairs=24, batch=2, epochs=4, lr=3e-3, mu=0.001, gate_systems=2, seed=11)
        T.tmamg_nn_init(lat.ctx, 7)
        rep = T.tmamg_nn_train(lat.ctx, T.tmamg_default_nn_params(window=4, **kw))
        assert rep.loss_last < rep.loss_first, (rep.loss_first, rep.loss_last)
        w_win = T.tmamg_nn_get_weights(lat.ctx)
        out = []
        for window in (0, 12):
            T.tmamg_nn_init(lat.ctx, 7)
            T.tmamg_nn_train(lat.ctx, T.tmamg_default_nn_params(window=window, **kw))
            out.append(T.tmamg_nn_get_weights(lat.ctx))
        assert np.array_equal(out[0], out[1])
        assert not np.array_equal(out[0], w_win)
    finally:
        lat.close()

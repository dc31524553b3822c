"""Gauge-covariant parallel-transport network in FP64 (oracle; test infrastructure only).

The learned preconditioner step is not in the paper; the method description adds it as an
extra fine-level preconditioner inside FGMRES. Readings:
  * three linear layers (no activation) with 4 -> 8 -> 8 -> 4 complex channels, each channel
    a colour 3-vector per site (the 12 = 4 x 3 spinor components enter as 4 channels);
  * a layer is out_a(x) = sum_h sum_b W_h[a, b] (T_h in_b)(x) over the nine hops
    h = 0 (T_0 = identity), h = 1 + 2 nu: (T in)(x) = U_nu(x) in(x + nu),
    h = 2 + 2 nu: (T in)(x) = U_nu(x - nu)^+ in(x - nu), with the fermion boundary phase;
  * the loss of a batch is sum_i |N(r_i) - e_i|^2 / |e_i|^2.
Complex gradients follow the convention grad = dL/dRe + i dL/dIm, so that
dL = Re(conj(grad) dW) and gradient descent is W <- W - lr grad.

Field layout: [..., T, Z, Y, X, channels, 3].
"""
import numpy as np

from . import dirac

CHANNELS = (4, 8, 8, 4)
NHOP = 9


def opposite(h):
    return 0 if h == 0 else (h + 1 if h % 2 == 1 else h - 1)


class Transport:
    """The nine parallel transports T_h of one gauge field."""

    def __init__(self, U, bc_t=-1):
        self.U = np.asarray(U, dtype=np.complex128)
        self.bc_t = bc_t
        self.Ubwd = [dirac.dag(dirac.link_shift(self.U[..., nu, :, :], [(-1 if d == nu else 0) for d in range(4)]))
                     for nu in range(4)]

    def apply(self, f, h):
        """T_h f for f [..., T, Z, Y, X, ch, 3]."""
        if h == 0:
            return f
        nu = (h - 1) // 2
        if h % 2 == 1:
            fs = dirac.shift_fwd(f, nu, self.bc_t)
            return np.einsum("...ab,...kb->...ka", self.U[..., nu, :, :], fs)
        fs = dirac.shift_bwd(f, nu, self.bc_t)
        return np.einsum("...ab,...kb->...ka", self.Ubwd[nu], fs)

    def adjoint(self, f, h):
        """T_h^+ f = T_opposite(h) f (the boundary phase is real)."""
        return self.apply(f, opposite(h))


def layer(tr: Transport, W, x):
    """out_a = sum_h sum_b W[h, a, b] (T_h x_b); W [9, cout, cin]."""
    out = 0
    for h in range(NHOP):
        out = out + np.einsum("ab,...bc->...ac", W[h], tr.apply(x, h))
    return out


def layer_backward(tr: Transport, W, x, g):
    """Gradients of a layer given g = grad wrt its output: (grad wrt W, grad wrt x)."""
    gW = np.zeros_like(W)
    gx = 0
    for h in range(NHOP):
        z = tr.apply(x, h)
        # grad W_h[a, b] = sum_{sites, colour, batch} g_a conj(z_b)
        gf = g.reshape((-1,) + g.shape[-2:])
        zf = np.conj(z).reshape((-1,) + z.shape[-2:])
        gW[h] = np.einsum("nac,nbc->ab", gf, zf)
        # grad x = sum_h T_h^+ (W_h^+ g)
        gx = gx + tr.adjoint(np.einsum("ba,...bc->...ac", np.conj(W[h]), g), h)
    return gW, gx


def init_weights(seed=1, scale=0.1, identity=True):
    """Identity-like start (W_0 embeds / projects the 4 input channels) plus small noise."""
    import synth
    Ws = []
    for l in range(3):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        W = synth.complex_normal(seed, 700 + l, (NHOP, cout, cin), var=1.0) * scale / np.sqrt(NHOP * cin)
        if identity:
            W[0] += np.eye(cout, cin)
        Ws.append(W)
    return Ws


def forward(tr: Transport, Ws, r):
    """N(r) for r [..., T, Z, Y, X, 4, 3]; returns the output and the layer inputs."""
    xs = [r]
    x = r
    for W in Ws:
        x = layer(tr, W, x)
        xs.append(x)
    return x, xs


def loss_and_grad(tr: Transport, Ws, r, e):
    """Batch loss sum_i |N(r_i) - e_i|^2 / |e_i|^2 and its gradients (r, e: [B, ..., 4, 3])."""
    y, xs = forward(tr, Ws, r)
    d = y - e
    axes = tuple(range(1, r.ndim))
    en = np.sum(np.abs(e) ** 2, axis=axes)
    loss = float(np.sum(np.sum(np.abs(d) ** 2, axis=axes) / en))
    g = 2.0 * d / en.reshape((-1,) + (1,) * (r.ndim - 1))
    grads = [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        grads[l], g = layer_backward(tr, Ws[l], xs[l], g)
    return loss, grads

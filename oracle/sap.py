"""Red-black Schwarz alternating procedure (SAP) in FP64 (oracle; test infrastructure only).

Paper Sec. 2: the lattice is divided into small blocks in a chessboard manner
and the local Dirac operators on the blocks are (approximately) inverted, red
blocks first, then black; SAP damps the high modes of the error.

Readings where the paper is silent:
  * colour of a block = parity of the sum of its block coordinates; red = even;
  * the block operator D_B keeps only hops whose two ends lie in the same block
    (Dirichlet boundary); the block solve is `mr_steps` steps of the minimal
    residual iteration on D_B from a zero start;
  * one SAP cycle = red sweep then black sweep, each using the residual
    recomputed from scratch; `cycles` cycles; SAP acts as a smoother that maps
    a residual r to a correction e (zero start).
"""
import numpy as np

from . import dirac


def block_index(L, bs):
    """Block coordinates of every site: int array [Lt, Lz, Ly, Lx, 4] (x, y, z, t order)."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return np.stack([x // bs[0], y // bs[1], z // bs[2], t // bs[3]], axis=-1)


def block_id(L, bs):
    """Linear block id of every site [Lt, Lz, Ly, Lx] and the block count."""
    bc = block_index(L, bs)
    nb = [L[d] // bs[d] for d in range(4)]
    bid = ((bc[..., 3] * nb[2] + bc[..., 2]) * nb[1] + bc[..., 1]) * nb[0] + bc[..., 0]
    return bid, int(np.prod(nb))


def block_colour(L, bs):
    """0 (red) or 1 (black) per site."""
    return block_index(L, bs).sum(axis=-1) % 2


class BlockOperator:
    """Block-diagonal part of D: every hop that leaves its block is dropped."""

    def __init__(self, op: dirac.Operator, bs):
        self.op = op
        self.bs = tuple(bs)
        L = op.L
        self.bid, self.nblocks = block_id(L, bs)
        self.colour = block_colour(L, bs)
        # keep[nu][sign] is 1 where the hop s -> s + sign*nu stays in the block
        self.keep_fwd = []
        self.keep_bwd = []
        for nu in range(4):
            ax = {0: 3, 1: 2, 2: 1, 3: 0}[nu]
            nb_f = np.roll(self.bid, -1, axis=ax)
            nb_b = np.roll(self.bid, 1, axis=ax)
            self.keep_fwd.append((nb_f == self.bid).astype(np.float64)[..., None, None])
            self.keep_bwd.append((nb_b == self.bid).astype(np.float64)[..., None, None])

    def apply(self, x, mu):
        op = self.op
        y = op.apply_local(x) + op.apply_twist(x, mu)
        for nu in range(4):
            y = y + self.keep_fwd[nu] * op.hop_fwd(x, nu) + self.keep_bwd[nu] * op.hop_bwd(x, nu)
        return y

    def block_dot(self, a, b):
        """<a, b> restricted to each block: [..., nblocks] complex."""
        prod = np.sum(np.conj(a) * b, axis=(-1, -2))  # [..., T, Z, Y, X]
        lead = prod.shape[:-4]
        flat = prod.reshape(lead + (-1,))
        ids = self.bid.ravel()
        out = np.zeros(lead + (self.nblocks,), dtype=np.complex128)
        for idx in np.ndindex(*lead) if lead else [()]:
            out[idx] = np.bincount(ids, weights=flat[idx].real, minlength=self.nblocks) + \
                1j * np.bincount(ids, weights=flat[idx].imag, minlength=self.nblocks)
        return out

    def per_site(self, v):
        """Broadcast a per-block value [..., nblocks] to sites [..., T, Z, Y, X, 1, 1]."""
        return v[..., self.bid][..., None, None]


def mr_block_solve(bop: BlockOperator, r, mu, colour, steps):
    """Minimal-residual steps on D_B for all blocks of one colour at once.

    Returns (e, rho): the correction (zero outside the colour) and the final
    block residual r_B - D_B e_B.
    """
    mask = (bop.colour == colour).astype(np.float64)[..., None, None]
    rho = r * mask
    e = np.zeros_like(r)
    for _ in range(steps):
        q = bop.apply(rho, mu) * mask
        qq = bop.block_dot(q, q).real
        qr = bop.block_dot(q, rho)
        alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
        a = bop.per_site(alpha)
        e = e + a * rho
        rho = rho - a * q
    return e, rho


def sap(op: dirac.Operator, r, mu, bs, cycles=2, mr_steps=3, bop=None):
    """SAP smoother: e ~ D(mu)^{-1} r, zero start. r may carry leading system axes (mu matching)."""
    if bop is None:
        bop = BlockOperator(op, bs)
    e = np.zeros_like(r)
    for _ in range(cycles):
        for colour in (0, 1):
            res = r - op.apply(e, mu)
            de, _ = mr_block_solve(bop, res, mu, colour, mr_steps)
            e = e + de
    return e

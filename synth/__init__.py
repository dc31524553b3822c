"""Seeded synthetic inputs for the multi-rhs / multi-shift twisted-mass solver.

This module is the only code shared by the CPU oracle and the CUDA path. It
holds none of the method's arithmetic: it draws random numbers and turns them
into workload data (gauge links, right-hand sides, shift lists, random start
vectors for the multigrid setup). Everything here is deterministic in
(seed, stream) and portable across machines: the random numbers come from a
counter-based splitmix64 generator written out below, not from a library RNG.

Array conventions (shared by every consumer):
  * lattice extents L = (Lx, Ly, Lz, Lt); site order lexicographic with x fastest,
    so a field has numpy shape [Lt, Lz, Ly, Lx, ...];
  * gauge field U: complex128 [Lt, Lz, Ly, Lx, 4, 3, 3], direction index 0..3 = x, y, z, t;
  * spinor field: complex128 [Lt, Lz, Ly, Lx, 4, 3] (spin, colour), a batch of
    them carries a leading system axis.

Gauge recipe (workload prep, not the method): U = exp(i eps H) with H a
Gaussian traceless Hermitian 3x3 matrix, reunitarised to SU(3).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) applied to a uint64 counter array."""
    with np.errstate(over="ignore"):
        z = counter * _GOLDEN + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _stream_base(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        key = _splitmix64(np.array([np.uint64(seed) ^ (np.uint64(stream) << np.uint64(40))],
                                   dtype=np.uint64))[0]
    return key


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in (0, 1], counter-based: element i = splitmix64(key + i) >> 11, scaled."""
    base = _stream_base(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(n, dtype=np.uint64) + base
    bits = _splitmix64(ctr) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform of two uniform streams."""
    m = (n + 1) // 2
    u = uniform(seed, stream, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[:m]))
    th = 2.0 * np.pi * u[m:]
    z = np.concatenate([r * np.cos(th), r * np.sin(th)])
    return z[:n]


def _uniform_at(base: np.uint64, idx: np.ndarray) -> np.ndarray:
    """The uniform() values at counter offsets idx of a stream."""
    with np.errstate(over="ignore"):
        ctr = idx.astype(np.uint64) + base
    bits = _splitmix64(ctr) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def _complex_normal_range(seed: int, stream: int, n: int, k0: int, k1: int, var: float) -> np.ndarray:
    """Elements [k0, k1) of complex_normal(seed, stream, (n,), var), computed alone. In
    normal(seed, stream, 2 n) the Box-Muller pair j takes its radius from uniform index j and its
    angle from index n + j, and gives z[j] = r cos(th), z[n + j] = r sin(th); complex element k is
    z[k] + i z[n + k]. Same arithmetic as the whole-array form, so any split gives the same numbers."""
    base = _stream_base(seed, stream)
    k = np.arange(k0, k1, dtype=np.int64)
    u_r = _uniform_at(base, k)
    u_t = _uniform_at(base, k + n)
    r = np.sqrt(-2.0 * np.log(u_r))
    th = 2.0 * np.pi * u_t
    sc = np.sqrt(var / 2.0)
    return (r * np.cos(th)) * sc + 1j * ((r * np.sin(th)) * sc)


def _parallel_rows(n: int, fn, chunk: int = 1 << 20):
    """Apply fn(k0, k1) over [0, n) in chunks on a thread pool (numpy releases the GIL in its
    loops), returning the concatenation in order."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    bounds = [(a, min(a + chunk, n)) for a in range(0, n, chunk)]
    if len(bounds) <= 1:
        return fn(0, n)
    workers = max(1, min(len(bounds), os.cpu_count() or 1, 32))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        parts = list(ex.map(lambda b: fn(*b), bounds))
    return np.concatenate(parts)


def complex_normal(seed: int, stream: int, shape, var: float = 1.0) -> np.ndarray:
    """Complex Gaussian with E|z|^2 = var (real and imaginary parts each var/2)."""
    n = int(np.prod(shape))
    if n <= (1 << 20):
        z = normal(seed, stream, 2 * n) * np.sqrt(var / 2.0)
        return (z[:n] + 1j * z[n:]).reshape(shape)
    return _parallel_rows(n, lambda a, b: _complex_normal_range(seed, stream, n, a, b, var)).reshape(shape)


def lattice_shape(L):
    Lx, Ly, Lz, Lt = (int(v) for v in L)
    return (Lt, Lz, Ly, Lx)


def _links(seed: int, eps: float, nlink: int, a: int, b: int) -> np.ndarray:
    """Links [a, b) of the recipe below: their Gaussian matrices are elements [9 a, 9 b) of the
    stream, so every split of the links gives the same field."""
    A = _complex_normal_range(seed, 101, 9 * nlink, 9 * a, 9 * b, 1.0).reshape(b - a, 3, 3)
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)
    lam, Q = np.linalg.eigh(H)
    ph = np.exp(1j * eps * lam)
    return reunitarise((Q * ph[:, None, :]) @ np.conj(np.swapaxes(Q, -1, -2)))


def gauge_field(L, eps: float, seed: int = 1, chunk: int = 1 << 17, processes: int | None = None) -> np.ndarray:
    """Random SU(3) links U = exp(i eps H), reunitarised.

    H = (A + A^dagger)/2 - tr/3 with A complex Gaussian entries (Re, Im each of
    variance 1/2); the exponential is taken through the eigendecomposition of H.
    Returns complex128 [Lt, Lz, Ly, Lx, 4, 3, 3].

    Large fields are made in chunks of `chunk` links on a pool of spawned processes (by default
    one per core when there are more than 16 chunks); the result does not depend on the split.
    """
    import os
    shp = lattice_shape(L) + (4,)
    nlink = int(np.prod(shp))
    bounds = [(a, min(a + chunk, nlink)) for a in range(0, nlink, chunk)]
    if processes is None:
        processes = (os.cpu_count() or 1) if len(bounds) > 16 else 1
    if processes <= 1 or len(bounds) == 1:
        U = np.concatenate([_links(seed, eps, nlink, a, b) for a, b in bounds])
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        U = np.empty((nlink, 3, 3), dtype=np.complex128)
        with ProcessPoolExecutor(max_workers=min(processes, len(bounds)),
                                 mp_context=mp.get_context("spawn")) as ex:
            futs = [(a, b, ex.submit(_links, seed, eps, nlink, a, b)) for a, b in bounds]
            for a, b, f in futs:
                U[a:b] = f.result()
    return U.reshape(shp + (3, 3))


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1; row 2 = conj(row0 x row1), so det U = 1."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def unit_gauge(L) -> np.ndarray:
    """The free field: every link the 3x3 identity."""
    shp = lattice_shape(L) + (4,)
    return np.broadcast_to(np.eye(3, dtype=np.complex128), shp + (3, 3)).copy()


def random_su3(n: int, seed: int, stream: int = 303, eps: float = 2.0) -> np.ndarray:
    """n random SU(3) matrices (for gauge transformations); complex128 [n, 3, 3]."""
    A = complex_normal(seed, stream, (n, 3, 3), var=1.0)
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)
    lam, Q = np.linalg.eigh(H)
    U = np.einsum("nab,nb,ncb->nac", Q, np.exp(1j * eps * lam), np.conj(Q))
    return reunitarise(U)


def gaussian_spinors(L, nvec: int, seed: int, stream: int = 202) -> np.ndarray:
    """nvec complex Gaussian spinor fields, complex128 [nvec, Lt, Lz, Ly, Lx, 4, 3]."""
    return complex_normal(seed, stream, (nvec,) + lattice_shape(L) + (4, 3), var=1.0)


def gaussian_coarse(Lc, nvec: int, d: int, seed: int, stream: int = 206) -> np.ndarray:
    """nvec complex Gaussian vectors of a coarse level with d unknowns per chirality,
    complex128 [nvec, Ltc, Lzc, Lyc, Lxc, 2, d]."""
    return complex_normal(seed, stream, (nvec,) + lattice_shape(Lc) + (2, d), var=1.0)


def z2_spinors(L, nvec: int, seed: int, stream: int = 204) -> np.ndarray:
    """Complex Z2 noise: each component (+-1 +- i)/sqrt(2), signs from the generator."""
    shape = (nvec,) + lattice_shape(L) + (4, 3)
    n = int(np.prod(shape))
    u = uniform(seed, stream, 2 * n)
    re = np.where(u[:n] < 0.5, -1.0, 1.0)
    im = np.where(u[n:] < 0.5, -1.0, 1.0)
    return ((re + 1j * im) / np.sqrt(2.0)).reshape(shape)


def point_sources(L, site=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 point sources e_{spin,colour} at one site (x, y, z, t); complex128 [12, ...]."""
    shape = (12,) + lattice_shape(L) + (4, 3)
    b = np.zeros(shape, dtype=np.complex128)
    x, y, z, t = site
    for s in range(4):
        for c in range(3):
            b[s * 3 + c, t, z, y, x, s, c] = 1.0
    return b


def log_shifts(n: int, lo: float = 1e-3, hi: float = 1e-1) -> np.ndarray:
    """n twisted masses log-spaced from lo to hi inclusive."""
    if n == 1:
        return np.array([lo])
    return lo * (hi / lo) ** (np.arange(n) / (n - 1))

"""Krylov solvers in FP64 (oracle; test infrastructure only).

* fgmres: flexible GMRES(m) with right preconditioning (the top-level and
  coarse-level solver of the method, paper Sec. 4: "a three-level AMG with a
  FGMRES solver at the top level", non-block FGMRES at the coarse levels).
  Arnoldi by modified Gram-Schmidt, the small least-squares problem by a
  library least-squares routine.
* block_gmres: block GMRES(m) (paper Sec. 4, block Krylov solvers at the
  coarsest level). Block Arnoldi with one pass of classical Gram-Schmidt over
  the previous blocks (the paper found CGS without re-orthogonalisation to
  perform best), a QR factorisation of each new block, and the block
  least-squares problem min ||E1 R0 - H Y||_F solved by a library routine.
  Inexact breakdown detection is not used (the paper leaves it out).

Vectors are flat complex128 arrays; operators are callables.
"""
import numpy as np


def _dot(a, b):
    return np.vdot(a, b)


def fgmres(A, b, tol=1e-10, restart=10, maxiter=1000, M=None, x0=None):
    """Solve A x = b to ||b - A x|| <= tol ||b||.

    Returns (x, info) with info = dict(iters, restarts, resid (true, relative), converged).
    M (optional) is a right preconditioner applied as z_j = M(v_j); it may vary
    from call to call (flexible variant: Z is stored).
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    n = b.size
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), dict(iters=0, restarts=0, resid=0.0, converged=True)
    total = 0
    restarts = 0
    r = b - A(x)
    beta = np.linalg.norm(r)
    while total < maxiter:
        if beta <= tol * bnorm:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        k = 0
        for j in range(restart):
            z = V[j] if M is None else np.asarray(M(V[j])).ravel()
            Z.append(z)
            w = A(z)
            for i in range(j + 1):
                H[i, j] = _dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            total += 1
            e1 = np.zeros(k + 1, dtype=np.complex128)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
            est = np.linalg.norm(e1 - H[:k + 1, :k] @ y)
            if est <= tol * bnorm or H[j + 1, j] == 0.0 or total >= maxiter:
                break
            V.append(w / H[j + 1, j])
        x = x + np.array(Z[:k]).T @ y
        r = b - A(x)
        beta = np.linalg.norm(r)
        restarts += 1
    res = beta / bnorm
    return x, dict(iters=total, restarts=restarts, resid=res, converged=bool(res <= tol))


def block_gmres(A, B, tol=1e-10, restart=10, maxiter=1000, X0=None, A_block=None):
    """Block GMRES(m) for A X = B, B of shape [n, s].

    A acts on one vector; A_block (optional) acts on an [n, s] block at once.
    Stops when every column j has ||B_j - A X_j|| <= tol ||B_j||.
    Returns (X, info) with info = dict(iters (block steps), resid [s], converged).
    """
    B = np.asarray(B, dtype=np.complex128)
    n, s = B.shape
    if A_block is None:
        def A_block(W):
            return np.stack([A(W[:, c]) for c in range(W.shape[1])], axis=1)
    X = np.zeros((n, s), dtype=np.complex128) if X0 is None else np.array(X0, dtype=np.complex128)
    bn = np.linalg.norm(B, axis=0)
    bn = np.where(bn == 0.0, 1.0, bn)
    total = 0
    R = B - A_block(X)
    while total < maxiter:
        if np.all(np.linalg.norm(R, axis=0) <= tol * bn):
            break
        V0, R0 = np.linalg.qr(R)
        Vs = [V0]
        H = np.zeros(((restart + 1) * s, restart * s), dtype=np.complex128)
        k = 0
        Y = None
        for j in range(restart):
            W = A_block(Vs[j])
            # one pass of classical Gram-Schmidt against all previous blocks
            Hij = [Vi.conj().T @ W for Vi in Vs]
            for i, Vi in enumerate(Vs):
                H[i * s:(i + 1) * s, j * s:(j + 1) * s] = Hij[i]
            for i, Vi in enumerate(Vs):
                W = W - Vi @ Hij[i]
            Q, Rn = np.linalg.qr(W)
            H[(j + 1) * s:(j + 2) * s, j * s:(j + 1) * s] = Rn
            k = j + 1
            total += 1
            E = np.zeros(((k + 1) * s, s), dtype=np.complex128)
            E[:s, :] = R0
            Hk = H[:(k + 1) * s, :k * s]
            Y, *_ = np.linalg.lstsq(Hk, E, rcond=None)
            est = np.linalg.norm(E - Hk @ Y, axis=0)
            if np.all(est <= tol * bn) or total >= maxiter:
                break
            Vs.append(Q)
        X = X + np.concatenate(Vs[:k], axis=1) @ Y
        R = B - A_block(X)
    res = np.linalg.norm(R, axis=0) / bn
    return X, dict(iters=total, resid=res, converged=bool(np.all(res <= tol)))

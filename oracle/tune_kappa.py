"""Kappa tuning for the synthetic workloads (workload preparation; oracle only).

Recipe of the precision-form and batched workloads: kappa is raised by bisection until the
smallest singular value of the Wilson-clover operator D_W (twisted mass 0) is about 1e-3 of
the largest. Singular values of D_W are the absolute eigenvalues of the Hermitian
H = gamma5 D_W, i.e. the square roots of the eigenvalues of D_W^+ D_W; both ends are taken
by Lanczos (scipy eigsh) on D_W^+ D_W applied through the FP64 oracle operator.

Reading: the bisection runs on an 8^3 x 16 lattice built with the same gauge
recipe (eps, seed) as the large lattice, because the numpy oracle cannot afford Lanczos on
the large volumes; the kappa found is used on the large lattice. The bisection stays below
the first kappa where sigma_min turns up again (critical point of a rough field).

python -m oracle.tune_kappa   -> writes tests/golden/kappa.json
"""
import json
import os
import sys
import time

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import dirac  # noqa: E402


def singular_extremes(op, tol=1e-3):
    shp = op.U.shape[:4] + (4, 3)
    n = int(np.prod(shp))

    def mv(v):
        x = v.reshape(shp)
        return op.apply_dagger(op.apply(x, 0.0), 0.0).ravel()

    A = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    v0 = synth.complex_normal(5, 9, (n,))
    lmax = eigsh(A, k=1, which="LA", tol=1e-3, v0=v0, return_eigenvectors=False)[0]
    lmin = eigsh(A, k=1, which="SA", tol=tol, v0=v0, ncv=40, maxiter=20000, return_eigenvectors=False)[0]
    return np.sqrt(max(lmin, 0.0)), np.sqrt(lmax)


def tune(L, eps, seed, c_sw=1.0, target=1e-3, lo=0.120, hi=0.150, npts=16, steps=6, log=print):
    """Scan kappa on [lo, hi]; if the ratio crosses the target before its minimum, bisect that
    crossing; otherwise take the kappa of the smallest ratio (closest approach to kappa_c)."""
    U = synth.gauge_field(L, eps, seed=seed)
    hist = []

    def ratio(k):
        t = time.time()
        smin, smax = singular_extremes(dirac.Operator(U, k, c_sw))
        r = smin / smax
        hist.append(dict(kappa=float(k), sigma_min=float(smin), sigma_max=float(smax), ratio=float(r),
                         seconds=time.time() - t))
        log(f"  kappa {k:.6f}: sigma_min {smin:.4e} sigma_max {smax:.4f} ratio {r:.3e} ({time.time() - t:.0f} s)",
            flush=True)
        return r

    grid = np.linspace(lo, hi, npts)
    rs = []
    for k in grid:
        rs.append(ratio(k))
        if rs[-1] < target:
            break
        if len(rs) >= 3 and rs[-1] > rs[-2] > rs[-3]:
            break  # past the minimum: sigma_min grows again beyond kappa_c
    rs = np.array(rs)
    if rs[-1] < target and len(rs) > 1:
        a, b = grid[len(rs) - 2], grid[len(rs) - 1]
        for _ in range(steps):
            m = 0.5 * (a + b)
            if ratio(m) > target:
                a = m
            else:
                b = m
        cand = [h for h in hist if h["kappa"] <= b]
        best = min(cand, key=lambda h: abs(np.log(h["ratio"] / target)))
        how = "target crossing"
    else:
        i = int(np.argmin(rs))
        a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(rs) - 1)]
        for _ in range(steps):  # golden-section-like refinement of the minimum
            m1, m2 = a + (b - a) / 3, b - (b - a) / 3
            if ratio(m1) < ratio(m2):
                b = m2
            else:
                a = m1
        best = min(hist, key=lambda h: h["ratio"])
        how = "minimum of sigma_min/sigma_max (target not reached)"
    return dict(kappa=float(best["kappa"]), ratio=float(best["ratio"]), history=hist, how=how)


def main():
    out_path = os.path.join(ROOT, "tests", "golden", "kappa.json")
    table = json.load(open(out_path)) if os.path.exists(out_path) else {}
    Ltune = (8, 8, 8, 16)
    jobs = [((16, 16, 16, 32), 0.25, 1), ((24, 24, 24, 48), 0.25, 1), ((32, 32, 32, 64), 0.2, 1),
            ((40, 40, 40, 80), 0.2, 1)]
    only = [float(a) for a in sys.argv[1:]]
    if only:  # tune a subset of gauge recipes (eps values); entries are merged into the table
        jobs = [j for j in jobs if j[1] in only]
    done = {}
    for Lbig, eps, seed in jobs:
        key = f"{Lbig[0]}x{Lbig[1]}x{Lbig[2]}x{Lbig[3]}_eps{eps}_seed{seed}"
        if (eps, seed) not in done:
            print(f"tuning eps={eps} seed={seed} on {Ltune}")
            done[(eps, seed)] = tune(Ltune, eps, seed)
        res = done[(eps, seed)]
        table[key] = dict(kappa=res["kappa"], ratio_on_tuning_lattice=res["ratio"],
                          tuning_lattice=list(Ltune), eps=eps, seed=seed, c_sw=1.0, target_ratio=1e-3,
                          method="bisection on sigma_min/sigma_max of D_W via Lanczos on D_W^+ D_W (oracle, FP64)",
                          outcome=res["how"],
                          history=res["history"])
        json.dump(table, open(out_path, "w"), indent=1)
    print("wrote", out_path)


if __name__ == "__main__":
    main()

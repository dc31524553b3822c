"""Benchmark of the multi-rhs / multi-shift twisted-mass solver on one GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--what solve|dirac]

Workload (precision form): 16^3 x 32 lattice, U = exp(i 0.25 H) reunitarised, c_sw = 1,
kappa from the tuning table in tests/golden/kappa.json (sigma_min / sigma_max of D_W ~ 1e-3),
mu = 0.003, 12 point-source right-hand sides; synthetic, seeded.

One JSON line on rank 0. Under torchrun (N > 1) every rank runs an independent replica of
the workload (the systems are independent; no data-path collective) and the time is the
maximum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = dict(name="precision-form 16^3x32, 12 point sources, mu=0.003", L=(16, 16, 16, 32), eps=0.25, c_sw=1.0,
                mu=0.003, nrhs=12, seed=1)
METRIC = "rhs x shift solves/s at FP64 rel. residual 1e-10; Dirac-op GB/s vs HBM peak"
DIRAC_WORKLOAD = "fine twisted-mass Wilson-clover stencil, 16^3x32, 12 systems (FP32 bundle)"


def kappa_for(L, eps, seed):
    path = os.path.join(ROOT, "tests", "golden", "kappa.json")
    key = f"{L[0]}x{L[1]}x{L[2]}x{L[3]}_eps{eps}_seed{seed}"
    if os.path.exists(path):
        tab = json.load(open(path))
        if key in tab:
            return float(tab[key]["kappa"]), "tuned"
    return 0.1335, "untuned"


def dirac_bytes_per_site(nsys, prec):
    """Algorithmic bytes of one fine stencil application per site: 4 links (18 reals), the
    clover blocks (72 reals), and every system's spinor read once and written once (24 reals each)."""
    es = 4 if prec == 32 else 8
    return (4 * 18 + 72) * es + nsys * 2 * 24 * es


# DRAM bytes (read + write) of one fine-stencil launch at 16^3x32 x 12 systems, from an ncu
# capture of that kernel; valid only for the kernel sources it was taken on (SHA-1 of dirac.cu
# and stencil.cuh), else reported as null
DIRAC_TRAFFIC = {"bytes": 237069824 + 120919040,
                 "sha1": {"dirac.cu": "24e92d0ad15242de099dc0789bc8e321b64cb249",
                          "stencil.cuh": "bdc68ee2e32fd9112f7efc57c95df0422ce387ff"}}


def dirac_traffic():
    import hashlib
    for name, want in DIRAC_TRAFFIC["sha1"].items():
        path = os.path.join(ROOT, "paper_2201_03872_gb300", "csrc", name)
        if not os.path.exists(path) or hashlib.sha1(open(path, "rb").read()).hexdigest() != want:
            return None
    return DIRAC_TRAFFIC["bytes"]


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region.

    The sampler starts before the warm-up (its start-up queries stay out of the timed region)
    and only the samples stamped inside mark()'s window are kept."""

    def __init__(self, idx):
        self.idx = idx
        self.proc = None
        self.path = None
        self.window = None

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __enter__(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "500"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            self.result = None
            return
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate()
        import datetime
        sm, smax, reasons = [], [], set()
        rows = []
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, f[1:]))
        if self.window is not None:
            inside = [r for r in rows if r[0] is not None and self.window[0] - 0.2 <= r[0] <= self.window[1] + 0.2]
            rows = inside or rows[-3:]
        for _, f in rows:
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        self.result = None if not sm else {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                                           "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(v, world):
    """The largest v over the ranks (NCCL on GPUs, or a gloo group on the host)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms):
    """Weak scaling: every rank processes units_per_rank units; the job's rate is all ranks' units
    over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- our arm
def run_dirac(args, world, rank, local):
    import torch
    from paper_2201_03872_gb300 import tmamg as T

    wl = WORKLOAD
    L = wl["L"]
    V = int(np.prod(L))
    nsys = wl["nrhs"]
    kappa, ksrc = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank)
    stream = torch.cuda.current_stream()
    ctx = T.tmamg_create(L, -1, stream.cuda_stream)
    T.tmamg_load_gauge(ctx, U)
    T.tmamg_set_operator(ctx, kappa, wl["c_sw"])
    mu = np.full(nsys, wl["mu"])
    x = synth.gaussian_spinors(L, nsys, seed=7 + rank).astype(np.complex64)
    nb = T.tmamg_bundle_bytes(ctx, nsys, 32)
    xf = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yf = torch.empty_like(xf)
    xb = torch.empty(nb // 4, dtype=torch.float32, device="cuda")
    yb = torch.empty_like(xb)
    T.tmamg_pack(ctx, xf, xb, nsys, 32)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        for _ in range(args.warmup):
            T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        h0 = time.time()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32)
            ev[k][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.time())
    total_ms = t0.elapsed_time(t1)
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    total_ms = max_over_ranks(total_ms, world)
    bytes_per_apply = dirac_bytes_per_site(nsys, 32) * V
    gbs = whole_job_rate(bytes_per_apply * args.steps, world, total_ms) / 1e9
    # end to end through the public API with host buffers: H2D of x, apply, D2H of y
    xh = torch.from_numpy(x.view(np.float32).copy()).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        xf.copy_(xh, non_blocking=True)
        T.tmamg_apply(ctx, xf, yf, nsys, mu, 32)
        yh.copy_(yf, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    T.tmamg_destroy(ctx)
    hbm, _, peak_src = read_peaks()
    achieved = bytes_per_apply / (kern_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": DIRAC_WORKLOAD,
                   "kappa": kappa, "kappa_source": ksrc, "nsys": nsys,
                   "l2": "working set 378 MB > 129 MB L2; back-to-back applications"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": dirac_traffic(), "peak_source": peak_src,
                     "kernel": "dirac_kernel<float,2>", "algorithmic_bytes_per_launch": bytes_per_apply},
        "e2e": {"value": whole_job_rate(bytes_per_apply * args.steps, world, e2e_ms) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(x.nbytes)},
        "gpu_launches": args.steps,
        "clocks": clk.result,
    }
    return line


def setup_kw():
    return dict(agg=(4, 4, 4, 4), nv=24, sap_block=(4, 4, 4, 4), sap_cycles=2, sap_mr_steps=3, setup_iters=20)


def solve_kw():
    return dict(tol=1e-10, restart=20, max_outer=40, coarse_tol=0.1, coarse_restart=40, coarse_maxiter=400)


def measure_dirac(T, ctx, nsys, mu, steps, stream):
    """CUDA-event time of the fine FP32 stencil on a bundle of nsys systems (same stream)."""
    import torch
    nb = T.tmamg_bundle_bytes(ctx, nsys, 32)
    xb = torch.randn(nb // 4, dtype=torch.float32, device="cuda")
    yb = torch.empty_like(xb)
    for _ in range(3):
        T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32)
        b.record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def run_solve(args, world, rank, local):
    import torch
    from paper_2201_03872_gb300 import tmamg as T

    wl = WORKLOAD
    L = wl["L"]
    V = int(np.prod(L))
    nrhs = wl["nrhs"]
    mus = [wl["mu"]]
    nsys = nrhs * len(mus)
    kappa, ksrc = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank)
    stream = torch.cuda.current_stream()
    ctx = T.tmamg_create(L, -1, stream.cuda_stream)
    T.tmamg_load_gauge(ctx, U)
    T.tmamg_set_operator(ctx, kappa, wl["c_sw"])
    t = time.time()
    T.tmamg_setup(ctx, T.setup_params(**setup_kw()))
    torch.cuda.synchronize()
    setup_s = time.time() - t
    b = synth.point_sources(L)
    bd = torch.from_numpy(b.view(np.float64).copy()).cuda()
    xd = torch.zeros(nsys * V * 24, dtype=torch.float64, device="cuda")
    sp = T.solve_params(**solve_kw())
    ok = True
    iters = None
    with Clocks(local) as clk:
        for _ in range(args.warmup):
            T.tmamg_solve(ctx, bd, nrhs, mus, len(mus), xd, 1, sp)
        torch.cuda.synchronize()
        barrier(world)
        launches0 = T.tmamg_kernel_launches()  # kernels launched before the timed region (ncu -s)
        torch.cuda.synchronize()
        h0 = time.time()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            rc, stats = T.tmamg_solve(ctx, bd, nrhs, mus, len(mus), xd, 1, sp)
            ok &= rc == 0 and all(s.status == 0 and s.true_rel_res <= 1e-10 for s in stats)
            iters = stats
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.time())
    launches = T.tmamg_kernel_launches() - launches0
    total_ms = max_over_ranks(t0.elapsed_time(t1), world)
    solves_per_s = whole_job_rate(nsys * args.steps, world, total_ms)
    # end to end through the public API with host buffers: b copied in, x copied out, every step
    bh = np.ascontiguousarray(b)
    xh = np.zeros((nrhs, len(mus)) + b.shape[1:], dtype=np.complex128)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(args.steps):
        T.tmamg_solve(ctx, bh, nrhs, mus, len(mus), xh, 0, sp)
    e2e_s = max_over_ranks(time.perf_counter() - t, world)
    # the fine stencil (dominant hot kernel named by the metric), same context and systems
    kern_ms = measure_dirac(T, ctx, nsys, np.full(nsys, wl["mu"]), 20, stream)
    variants = {}
    if args.variants:
        # same workload, other forms of the method (each timed over the same number of steps)
        def timed(label, nr, c=ctx, **kw):
            spv = T.solve_params(**dict(solve_kw(), **kw))
            T.tmamg_solve(c, bd, nr, mus, len(mus), xd, 1, spv)
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            okv = True
            for _ in range(args.steps):
                rcv, stv = T.tmamg_solve(c, bd, nr, mus, len(mus), xd, 1, spv)
                okv &= rcv == 0 and all(q.status == 0 for q in stv)
            z.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(z) / args.steps
            variants[label] = {"solves_per_s": nr * len(mus) / (ms * 1e-3), "ms_per_step": ms, "all_converged": okv,
                               "fgmres_iterations": stv[0].inner_iters, "coarse_iterations": stv[0].coarse_iters}
        def guarded(label, fn):
            # a variant that fails is recorded as such; the headline line is still printed
            try:
                fn()
            except Exception as exc:  # noqa: BLE001
                variants[label] = {"error": f"{type(exc).__name__}: {exc}"}

        guarded("single_system", lambda: timed("single_system", 1))
        # the plain comparator: one system, every vector, operator and reduction in FP64
        guarded("plain_fp64_single_system", lambda: timed("plain_fp64_single_system", 1, precision=64))
        guarded("block_gmres_coarse", lambda: timed("block_gmres_coarse", nrhs, coarse_solver=1))

        def three_level():
            # a second coarsening (2^4 aggregates of the 4^3 x 8 level-1 lattice, Nv = 32), the middle level
            # solved by FGMRES(10) to 7e-2 with the level-2 correction and 3 MR steps as its preconditioner
            ctx3 = T.tmamg_create(L, -1, stream.cuda_stream)
            try:
                T.tmamg_load_gauge(ctx3, U)
                T.tmamg_set_operator(ctx3, kappa, wl["c_sw"])
                t = time.time()
                T.tmamg_setup(ctx3, T.setup_params(levels=3, agg2=(2, 2, 2, 2), nv2=32, **setup_kw()))
                torch.cuda.synchronize()
                setup3 = time.time() - t
                timed("three_level", nrhs, c=ctx3)
                variants["three_level"]["setup_seconds"] = setup3
            finally:
                T.tmamg_destroy(ctx3)

        guarded("three_level", three_level)

        def learned_step():
            t = time.time()
            rep = T.tmamg_nn_train(ctx, T.tmamg_default_nn_params(pairs=48, batch=12, epochs=30, lr=2e-3,
                                                                  mu=wl["mu"], gate_systems=4))
            torch.cuda.synchronize()
            timed("learned_step", nrhs, use_nn=2)
            variants["learned_step"].update({"train_seconds": time.time() - t, "loss_first": rep.loss_first,
                                             "loss_last": rep.loss_last, "gate_iterations_plain": rep.iters_plain,
                                             "gate_iterations_with_step": rep.iters_nn,
                                             "gate_enabled": bool(rep.enabled)})

        guarded("learned_step", learned_step)
    T.tmamg_destroy(ctx)
    hbm, _, peak_src = read_peaks()
    bytes_per_apply = dirac_bytes_per_site(nsys, 32) * V
    achieved = bytes_per_apply / (kern_ms * 1e-3) / 1e9
    s0 = iters[0]
    line = {
        "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "lattice": "16^3x32", "systems_per_step": nsys, "kappa": kappa,
                   "kappa_source": ksrc, "c_sw": wl["c_sw"], "mu": wl["mu"], "tol": 1e-10,
                   "amg": "2-level, 4^4 aggregates, Nv=24, 20 setup iterations, SAP 4^4 blocks x 2 cycles x 3 MR, "
                          "FGMRES(20) + FP64 refinement, persistent coarse GMRES(40) to 0.1",
                   "setup_seconds": setup_s, "all_converged": bool(ok),
                   "iterations": {"outer": s0.outer_iters, "fgmres": s0.inner_iters, "coarse": s0.coarse_iters},
                   "l2": "working set > 129 MB L2 (solver vectors 3+ GB)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": dirac_traffic(), "peak_source": peak_src, "kernel": "dirac_kernel<float,2> (fine stencil)",
                     "algorithmic_bytes_per_launch": bytes_per_apply, "launch_ms": kern_ms},
        "e2e": {"value": whole_job_rate(nsys * args.steps, world, e2e_s * 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": int(bh.nbytes), "d2h_bytes_per_step": int(xh.nbytes)},
        "gpu_launches": int(launches),
        "launches_before_timed": int(launches0),
        "clocks": clk.result,
    }
    if variants:
        line["variants"] = variants
    return line


def cpu_solve_baseline(iters_per_solve=21, steps=0, warmup=0):
    """The FP64 numpy oracle on the same lattice: one fine-level AMG iteration (operator
    applications, SAP smoother, restriction and prolongation with a random P) for one system,
    timed on the host cores; solves/s = 1 / (time per iteration x iterations per solve), with
    the FGMRES iteration count of the GPU solver on this workload (21, or the count measured in
    the same run). Setup and the coarse solve are left out, so this over-estimates the CPU rate.
    With steps > 0 (the reference arm) the iteration is timed once to express it in oracle operator
    applications, then warmup + steps operator applications are timed one by one and the rate uses
    their mean, so that every step is a bounded sample (one application, about a second)."""
    from oracle import dirac, sap as osap, amg
    wl = WORKLOAD
    L = wl["L"]
    kappa, _ = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"])
    op = dirac.Operator(U, kappa, wl["c_sw"])
    x = synth.gaussian_spinors(L, 1, seed=7)[0]
    bop = osap.BlockOperator(op, (4, 4, 4, 4))
    Vt = synth.gaussian_spinors(L, 24, seed=8)
    P = amg.Prolongation(amg.FineLevel.to_chi(Vt), L, (4, 4, 4, 4))
    t = time.perf_counter()
    y = op.apply(x, wl["mu"])                       # the FGMRES operator application
    rc = P.restrict(amg.FineLevel.to_chi(y))
    e = amg.FineLevel.to_spin(P.prolong(rc))
    r2 = y - op.apply(e, wl["mu"])                  # residual for the smoother
    e = e + osap.sap(op, r2, wl["mu"], (4, 4, 4, 4), cycles=2, mr_steps=3, bop=bop)
    dt = time.perf_counter() - t
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if steps <= 0:
        return {"value": 1.0 / (dt * iters_per_solve), "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"one fine-level AMG iteration of the numpy FP64 oracle on 16^3x32 ({dt:.1f} s), times "
                          f"{iters_per_solve} iterations per solve; setup and coarse solves excluded"}
    t = time.perf_counter()
    op.apply(x, wl["mu"])
    per_iter = dt / (time.perf_counter() - t)  # one AMG iteration in operator applications
    times = []
    for k in range(warmup + steps):
        t = time.perf_counter()
        op.apply(x, wl["mu"])
        if k >= warmup:
            times.append(time.perf_counter() - t)
    t_op = float(np.mean(times))
    return {"value": 1.0 / (t_op * per_iter * iters_per_solve), "unit": "solves/s", "cores": cores,
            "kind": "oracle",
            "sample": f"numpy FP64 oracle on 16^3x32, one system: {warmup} + {steps} timed operator applications "
                      f"(mean {t_op:.2f} s) x {per_iter:.1f} applications per fine-level AMG iteration (one "
                      f"iteration timed, {dt:.1f} s: operator, restriction and prolongation with a random P, SAP) "
                      f"x {iters_per_solve} iterations per solve; setup and coarse solves excluded"}


def cpu_dirac_baseline(steps=0, warmup=0):
    """The FP64 oracle operator on the same lattice (4 systems), timed on the host cores: about 8 s
    of applications, or (the reference arm) warmup + steps applications timed one by one."""
    from oracle import dirac
    wl = WORKLOAD
    L = wl["L"]
    V = int(np.prod(L))
    kappa, _ = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"])
    op = dirac.Operator(U, kappa, wl["c_sw"])
    nsys = 4
    x = synth.gaussian_spinors(L, nsys, seed=7)
    mu = np.full(nsys, wl["mu"])
    op.apply(x[:1], mu[:1])
    if steps > 0:
        times = []
        for k in range(warmup + steps):
            t = time.perf_counter()
            op.apply(x, mu)
            if k >= warmup:
                times.append(time.perf_counter() - t)
        dt, reps = float(np.mean(times)), steps
    else:
        t = time.perf_counter()
        reps = 0
        while True:
            op.apply(x, mu)
            reps += 1
            if time.perf_counter() - t > 8.0:
                break
        dt = (time.perf_counter() - t) / reps
    gbs = dirac_bytes_per_site(nsys, 32) * V / dt / 1e9
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"numpy FP64 oracle D(mu) on 16^3x32 with {nsys} systems, {reps} applications; "
                      "bytes counted with the same FP32 algorithmic formula as the GPU line"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--what", default="solve", choices=["solve", "dirac"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the single-system, block-GMRES and learned-step forms")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init()
    if args.impl == "reference":
        if rank != 0:
            return
        cb = (cpu_solve_baseline(steps=args.steps, warmup=args.warmup) if args.what == "solve"
              else cpu_dirac_baseline(steps=args.steps, warmup=args.warmup))
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": cb["unit"], "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD["name"] if args.what == "solve" else
                           DIRAC_WORKLOAD},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    line = run_solve(args, world, rank, local) if args.what == "solve" else run_dirac(args, world, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = (cpu_solve_baseline(line["config"]["iterations"]["fgmres"]) if args.what == "solve"
                                    else cpu_dirac_baseline())
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

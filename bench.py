"""Benchmark of the multi-rhs / multi-shift twisted-mass solver on one GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--what solve|dirac]
                [--workload largest|batched|precision] [--no-variants] [--no-cpu-baseline]

Headline workload (largest single-GPU configuration): 40^3 x 80 lattice, U = exp(i 0.2 H)
reunitarised, c_sw = 1, kappa from the tuning table in tests/golden/kappa.json, 4 Gaussian
right-hand sides x 4 twisted masses {0.0015, 0.005, 0.015, 0.05} = 16 systems, three-level AMG
(4^4 aggregates with Nv = 24, then 2^4 aggregates with Nv = 32), FP32 fine level and SAP, FP16
coarse operators on the tensor cores, FP64 outer residuals; synthetic, seeded.
Variants over other workloads: the batched multi-shift form (24^3 x 48, 4 complex Z2-noise
right-hand sides x 10 log-spaced twisted masses = 40 systems in one solve) and the precision
form (16^3 x 32, 12 point sources), with the single-system, plain FP64, block-GMRES, three-level
and learned-step forms of the latter.

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

METRIC = "rhs x shift solves/s at FP64 rel. residual 1e-10; Dirac-op GB/s vs HBM peak"

_AMG2 = dict(levels=2, agg=(4, 4, 4, 4), nv=24, sap_block=(4, 4, 4, 4), sap_cycles=2, sap_mr_steps=3, setup_iters=20)
WORKLOADS = {
    "largest": dict(
        name="largest single-GPU: 40^3x80, eps 0.2, 4 Gaussian rhs x 4 twisted masses {0.0015,0.005,0.015,0.05}, "
             "3-level AMG",
        L=(40, 40, 40, 80), eps=0.2, c_sw=1.0, seed=1, nrhs=4, rhs="gaussian", mus=[0.0015, 0.005, 0.015, 0.05],
        setup=dict(_AMG2, levels=3, agg2=(2, 2, 2, 2), nv2=32, setup_gmres_steps=20, sap_mr_steps=6, setup_iters=40),
        solve=dict(tol=1e-10, restart=5, inner_cycles=4, max_outer=60, coarse_tol=0.2, coarse_restart=40,
                   coarse_maxiter=400, mid_tol=7e-2, mid_restart=10, mid_maxiter=50, mid_smooth=3,
                   sap_cycles=2, sap_mr_steps=4),
        amg="3-level: 4^4 aggregates Nv=24 (10^3x20 x 48), then 2^4 aggregates Nv=32 (5^3x10 x 64); 40 setup "
            "iterations; SAP 4^4 blocks x 2 cycles x 6 MR in the setup, x 4 MR in the solve; FGMRES(5) + FP64 "
            "refinement; middle FGMRES(10) to 7e-2 "
            "with 3 MR smoothing steps; bottom persistent GMRES(40) to 0.2; up to 4 FP32 FGMRES(5) cycles per FP64 "
            "residual"),
    "batched": dict(
        name="batched multi-shift: 24^3x48, eps 0.25, 4 complex Z2-noise rhs x 10 twisted masses log-spaced "
             "1e-3..1e-1 (40 systems)",
        L=(24, 24, 24, 48), eps=0.25, c_sw=1.0, seed=1, nrhs=4, rhs="z2", mus=list(synth.log_shifts(10)),
        setup=dict(_AMG2, sap_mr_steps=6),
        solve=dict(tol=1e-10, restart=10, inner_cycles=2, max_outer=60, coarse_tol=0.1, coarse_restart=40,
                   coarse_maxiter=400, sap_mr_steps=3),
        amg="2-level: 4^4 aggregates Nv=24 (6^3x12 x 48); 20 setup iterations; SAP 4^4 x 2 x 6 MR in the setup, "
            "x 3 MR in the solve; FGMRES(10) + "
            "FP64 refinement (up to 2 FP32 cycles per FP64 residual); persistent coarse GMRES(40) to 0.1"),
    "precision": dict(
        name="precision-form 16^3x32, 12 point sources, mu=0.003",
        L=(16, 16, 16, 32), eps=0.25, c_sw=1.0, seed=1, nrhs=12, rhs="point", mus=[0.003],
        setup=dict(_AMG2, sap_mr_steps=6),
        solve=dict(tol=1e-10, restart=20, max_outer=40, coarse_tol=0.1, coarse_restart=40, coarse_maxiter=400,
                   sap_mr_steps=4),
        amg="2-level: 4^4 aggregates Nv=24 (4^3x8 x 48); 20 setup iterations; SAP 4^4 x 2 x 6 MR in the setup, x 4 MR "
            "in the solve; FGMRES(20) + "
            "FP64 refinement; persistent coarse GMRES(40) to 0.1"),
    "learned": dict(
        name="learned-step form: 32^3x64, eps 0.2, 8 Gaussian rhs, mu=0.002",
        L=(32, 32, 32, 64), eps=0.2, c_sw=1.0, seed=1, nrhs=8, rhs="gaussian", mus=[0.002],
        setup=dict(_AMG2, sap_mr_steps=6),
        solve=dict(tol=1e-10, restart=10, inner_cycles=2, max_outer=60, coarse_tol=0.1, coarse_restart=40,
                   coarse_maxiter=400, sap_mr_steps=4),
        amg="2-level: 4^4 aggregates Nv=24 (8^3x16 x 48); 20 setup iterations; SAP 4^4 x 2 x 6 MR in the setup, "
            "x 4 MR in the solve; FGMRES(10) + FP64 refinement; persistent coarse GMRES(40) to 0.1"),
}
HEADLINE = "largest"
def dirac_workload(L, nsys):
    return "fine twisted-mass Wilson-clover stencil, %dx%dx%dx%d, %d systems (FP32 bundle)" % (tuple(L) + (nsys,))


def rhs_for(wl, rank=0):
    """The workload's right-hand sides, complex128 [nrhs, Lt, Lz, Ly, Lx, 4, 3]."""
    L, n = wl["L"], wl["nrhs"]
    if wl["rhs"] == "point":
        return synth.point_sources(L)[:n]
    if wl["rhs"] == "z2":
        return synth.z2_spinors(L, n, seed=11 + rank)
    return synth.gaussian_spinors(L, n, seed=11 + rank)


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


# DRAM bytes (read + write) of one launch of a kernel, from an ncu capture on a lattice whose
# working set is far larger than the L2 (24^3x48, 16 systems; the commands are in profiles/).
# The bytes of one launch grow with the lattice volume at a fixed system count, so a launch of
# the same kernel on another volume is reported as the captured bytes times the volume ratio.
# Valid only for the kernel sources the capture was taken on (SHA-1 of the files), else null.
KERNEL_TRAFFIC = {
    "dirac_f32": {"bytes": 1974789888 + 1003945472, "L": (24, 24, 24, 48), "nsys": 16,
                  "sha1": {"dirac.cu": "12f89d25e3a45b15f4f4277b40587ba3f9cd98b6",
                           "stencil.cuh": "bbe52b7b1bde87326034de584ba1950fba6a7d1b"}},
    "sap_mr": {"bytes": 3087883264 + 1500493824, "L": (24, 24, 24, 48), "nsys": 16,
               "sha1": {"sap.cu": "f57da3cd9bff38252df3a6da1a335eaf2ab9f83a",
                        "stencil.cuh": "bbe52b7b1bde87326034de584ba1950fba6a7d1b"}},
}


def kernel_traffic(kernel, L, nsys):
    """Captured DRAM bytes of one launch of `kernel` scaled to lattice L, or None (no capture for
    this system count, or the kernel's sources changed since the capture)."""
    import hashlib
    e = KERNEL_TRAFFIC.get(kernel)
    if e is None or e["nsys"] != nsys:
        return None
    for name, want in e["sha1"].items():
        path = os.path.join(ROOT, "paper_2201_03872_gb300", "csrc", name)
        if not os.path.exists(path) or hashlib.sha1(open(path, "rb").read()).hexdigest() != want:
            return None
    return int(e["bytes"] * float(np.prod(L)) / float(np.prod(e["L"])))


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

    wl = WORKLOADS[args.workload or "precision"]
    L = wl["L"]
    V = int(np.prod(L))
    nsys = args.nsys or wl["nrhs"]
    kappa, ksrc = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank)
    stream = torch.cuda.current_stream()
    ctx = T.tmamg_create(L, -1, stream.cuda_stream)
    T.tmamg_load_gauge(ctx, U)
    T.tmamg_set_operator(ctx, kappa, wl["c_sw"])
    mu = np.full(nsys, wl["mus"][0])
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
        "config": {"workload": dirac_workload(L, nsys),
                   "kappa": kappa, "kappa_source": ksrc, "nsys": nsys,
                   "l2": "working set %.0f MB > 129 MB L2; back-to-back applications" % (bytes_per_apply / 1e6)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": kernel_traffic("dirac_f32", L, nsys), "peak_source": peak_src,
                     "kernel": "dirac_kernel<float,2>", "algorithmic_bytes_per_launch": bytes_per_apply},
        "e2e": {"value": whole_job_rate(bytes_per_apply * args.steps, world, e2e_ms) / 1e9, "unit": "GB/s",
                "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": int(x.nbytes)},
        "gpu_launches": args.steps,
        "clocks": clk.result,
    }
    return line


def run_sap(args, world, rank, local):
    """The SAP smoother alone on the precision-form lattice with the largest workload's system count
    and SAP settings (diagnostic mode: one colour sweep pair per cycle), for profiling the block
    solver: per block and system tile it does the work of one SAP of that workload, so its DRAM
    traffic scales to it by the lattice volume."""
    import torch
    from paper_2201_03872_gb300 import tmamg as T
    wl = WORKLOADS[args.workload or "precision"]
    L = wl["L"]
    big = WORKLOADS[HEADLINE]
    nsys = args.nsys or big["nrhs"] * len(big["mus"])
    cyc, mr = big["setup"]["sap_cycles"], big["setup"]["sap_mr_steps"]
    kappa, _ = kappa_for(L, wl["eps"], wl["seed"])
    stream = torch.cuda.current_stream()
    ctx = T.tmamg_create(L, -1, stream.cuda_stream)
    T.tmamg_load_gauge(ctx, synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank))
    T.tmamg_set_operator(ctx, kappa, wl["c_sw"])
    nb = T.tmamg_bundle_bytes(ctx, nsys, 32)
    r0 = torch.randn(nb // 4, dtype=torch.float32, device="cuda")
    r = torch.empty_like(r0)
    e = torch.empty_like(r0)
    mu = np.full(nsys, wl["mus"][0])
    blk = wl["setup"]["sap_block"]
    for _ in range(args.warmup):
        r.copy_(r0)
        T.tmamg_sap(ctx, r, e, nsys, mu, blk, cyc, mr)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        r.copy_(r0)
        T.tmamg_sap(ctx, r, e, nsys, mu, blk, cyc, mr)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) * 1e3 / args.steps
    T.tmamg_destroy(ctx)
    return {"metric": "SAP smoother applications/s (diagnostic)", "value": 1e3 / ms, "unit": "applications/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "data": "synthetic", "config": {"workload": "SAP 4^4 blocks x %d cycles x %d MR on %dx%dx%dx%d, %d systems"
                                                     % ((cyc, mr) + tuple(L) + (nsys,))}}


def run_eo(args, world, rank, local):
    """The even-odd Schur complement operator M_ee alone (diagnostic mode): CUDA-event time per application
    against one full stencil application on the same bundle, and the site-local solve's own launch time."""
    import torch
    from paper_2201_03872_gb300 import tmamg as T
    wl = WORKLOADS[args.workload or "precision"]
    L = wl["L"]
    big = WORKLOADS[HEADLINE]
    nsys = args.nsys or big["nrhs"] * len(big["mus"])
    kappa, _ = kappa_for(L, wl["eps"], wl["seed"])
    stream = torch.cuda.current_stream()
    ctx = T.tmamg_create(L, -1, stream.cuda_stream)
    T.tmamg_load_gauge(ctx, synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank))
    T.tmamg_set_operator(ctx, kappa, wl["c_sw"])
    nb = T.tmamg_bundle_bytes(ctx, nsys, 32)
    xb = torch.randn(nb // 4, dtype=torch.float32, device="cuda")
    yb = torch.empty_like(xb)
    mu = np.full(nsys, wl["mus"][0])
    out = {}
    for name, fn in (("schur", lambda: T.tmamg_dirac_eo(ctx, xb, yb, nsys, mu, 32)),
                     ("dirac", lambda: T.tmamg_dirac(ctx, xb, yb, nsys, mu, 32))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        z.record(stream)
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(z) / args.steps
    T.tmamg_profile_enable(1)
    T.tmamg_dirac_eo(ctx, xb, yb, nsys, mu, 32)
    torch.cuda.synchronize()
    rec = T.tmamg_profile_report()
    T.tmamg_profile_enable(0)
    T.tmamg_destroy(ctx)
    ms = out["schur"]
    return {"metric": "even-odd Schur operator applications/s (diagnostic)", "value": 1e3 / ms,
            "unit": "applications/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "data": "synthetic", "dirac_ms": out["dirac"],
            "eo_solve_ms": rec.get("eo_solve", [0, 0.0])[1],
            "config": {"workload": "M_ee = A_ee - H_eo A_oo^-1 H_oe (two stencils + site solves) on %dx%dx%dx%d, "
                                   "%d systems, FP32" % (tuple(L) + (nsys,))}}


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
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    del xb, yb
    torch.cuda.empty_cache()
    return ms


class Problem:
    """A workload on the GPU: context with gauge field, operator and multigrid setup, and the
    right-hand sides and solution buffers on the device."""

    def __init__(self, wl, rank, stream, setup_overrides=None):
        import torch
        from paper_2201_03872_gb300 import tmamg as T
        self.T, self.wl, self.stream = T, wl, stream
        L = wl["L"]
        self.L, self.V = L, int(np.prod(L))
        self.nrhs, self.mus = wl["nrhs"], list(wl["mus"])
        self.nsys = self.nrhs * len(self.mus)
        self.kappa, self.ksrc = kappa_for(L, wl["eps"], wl["seed"])
        t = time.time()
        self.U = synth.gauge_field(L, wl["eps"], seed=wl["seed"] + rank)
        self.b = rhs_for(wl, rank)
        self.input_seconds = time.time() - t
        self.ctx = T.tmamg_create(L, -1, stream.cuda_stream)
        T.tmamg_load_gauge(self.ctx, self.U)
        T.tmamg_set_operator(self.ctx, self.kappa, wl["c_sw"])
        torch.cuda.synchronize()
        t = time.time()
        T.tmamg_setup(self.ctx, T.setup_params(**dict(wl["setup"], **(setup_overrides or {}))))
        torch.cuda.synchronize()
        self.setup_seconds = time.time() - t
        self.bd = torch.from_numpy(self.b.view(np.float64).copy()).cuda()
        self.xd = torch.zeros(self.nsys * self.V * 24, dtype=torch.float64, device="cuda")

    def params(self, **kw):
        return self.T.solve_params(**dict(self.wl["solve"], **kw))

    def solve(self, sp, nrhs=None):
        nr = self.nrhs if nrhs is None else nrhs
        rc, stats = self.T.tmamg_solve(self.ctx, self.bd, nr, self.mus, len(self.mus), self.xd, 1, sp)
        ok = rc == 0 and all(q.status == 0 and q.true_rel_res <= self.wl["solve"]["tol"] for q in stats)
        return ok, stats

    def close(self):
        self.T.tmamg_destroy(self.ctx)
        import torch
        del self.bd, self.xd
        torch.cuda.empty_cache()


def stats_summary(stats):
    s0 = stats[0]
    return {"outer": max(q.outer_iters for q in stats), "fgmres": max(q.inner_iters for q in stats),
            "coarse": s0.coarse_iters, "max_true_rel_res": max(q.true_rel_res for q in stats)}


def timed_solves(pb, sp, steps, stream, nrhs=None):
    """CUDA-event time of `steps` solves after one untimed solve; (ms per solve, converged, stats)."""
    import torch
    pb.solve(sp, nrhs)
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ok = True
    stats = None
    for _ in range(steps):
        okk, stats = pb.solve(sp, nrhs)
        ok &= okk
    z.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(z) / steps, ok, stats


FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2070 MHz
FP64_PEAK_TFLOPS = 1.25                                   # GB300 nominal FP64 (non-tensor)
DIRAC_FLOP_PER_SITE_SYSTEM = 1896                         # hops 1320 + clover 2 x 252 + twist/diag 48 + combine 24


def kernel_profile(pb, sp, stream):
    """One more solve with the library's per-kernel event timing on: {kernel: (launches, ms)} and the
    solve's own CUDA-event time."""
    import torch
    T = pb.T
    T.tmamg_profile_enable(1)
    try:
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ok, stats = pb.solve(sp)
        z.record(stream)
        torch.cuda.synchronize()
        rec = T.tmamg_profile_report()
    finally:
        T.tmamg_profile_enable(0)
    return rec, a.elapsed_time(z), stats


def kernel_rooflines(pb, rec, total_ms, stats):
    """Per-kernel time share of one profiled solve and, where an algorithmic count is defined, the
    achieved rate against its peak (HBM copy bandwidth, FP32 or FP64 ALU rate)."""
    hbm, _, peak_src = read_peaks()
    V, N = pb.V, pb.nsys
    st = pb.wl["setup"]
    nv = st["nv"]
    asz = int(np.prod(st["agg"]))
    steps = pb.wl["solve"].get("sap_mr_steps") or pb.wl["setup"].get("sap_mr_steps", 3)
    out = {}
    for name, (cnt, ms) in sorted(rec.items(), key=lambda kv: -kv[1][1]):
        e = {"launches": cnt, "ms": ms, "share": ms / total_ms, "ms_per_launch": ms / max(cnt, 1)}
        per = ms / max(cnt, 1) * 1e-3
        if name == "dirac_f32":
            b = dirac_bytes_per_site(N, 32) * V
            e.update(bound="hbm", algorithmic_bytes_per_launch=b, achieved=b / per / 1e9, peak=hbm, unit="GB/s")
        elif name == "residual_f64":
            f = DIRAC_FLOP_PER_SITE_SYSTEM * V * N
            e.update(bound="alu", algorithmic_flops_per_launch=f, achieved=f / per / 1e12, peak=FP64_PEAK_TFLOPS,
                     unit="TFLOP/s", peak_source="nominal GB300 FP64")
        elif name in ("restrict", "prolong"):
            # P (FP32 complex, 12 Nv per site) plus the fine vectors (FP32, 96 B per site and system)
            b = V * (12 * nv * 8 + 96 * N)
            e.update(bound="hbm", algorithmic_bytes_per_launch=b, achieved=b / per / 1e9, peak=hbm, unit="GB/s")
        elif name == "coarse_gmres":
            # the bottom level's operator stream per Arnoldi step: 5 stored n_c x n_c FP16 complex blocks
            # per coarse site (self + 4 forward hops; the backward hops follow by gamma5-hermiticity),
            # times the Arnoldi steps of one launch (the solve's bottom iterations over its launches)
            lv = st.get("levels", 2)
            Lc = [a // b for a, b in zip(pb.L, st["agg"])]
            nc = 2 * nv
            if lv == 3:
                Lc = [a // b for a, b in zip(Lc, st["agg2"])]
                nc = 2 * st["nv2"]
            steps_per_launch = stats[0].coarse_iters / max(cnt, 1)
            b = int(np.prod(Lc)) * 5 * nc * nc * 4 * steps_per_launch
            e.update(bound="hbm", algorithmic_bytes_per_launch=b, achieved=b / per / 1e9, peak=hbm, unit="GB/s",
                     arnoldi_steps_per_launch=steps_per_launch)
        elif name == "sap_mr":
            # one colour sweep: half the sites, `steps` block-operator applications per system
            f = DIRAC_FLOP_PER_SITE_SYSTEM * (V // 2) * N * steps
            e.update(bound="alu", algorithmic_flops_per_launch=f, achieved=f / per / 1e12,
                     peak=FP32_ALU_PEAK_TFLOPS, unit="TFLOP/s", peak_source="152 SMs x 128 FP32 lanes x 2 x 2070 MHz")
        if "achieved" in e:
            e["frac"] = e["achieved"] / e["peak"]
            e.setdefault("peak_source", peak_src)
            e["traffic"] = kernel_traffic(name, pb.L, N)
        out[name] = e
    return out


def run_solve(args, world, rank, local):
    import torch
    from paper_2201_03872_gb300 import tmamg as T

    wl = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    pb = Problem(wl, rank, stream)
    nsys, V = pb.nsys, pb.V
    sp = pb.params()
    ok = True
    stats = None
    with Clocks(local) as clk:
        for _ in range(args.warmup):
            pb.solve(sp)
        torch.cuda.synchronize()
        barrier(world)
        launches0 = T.tmamg_kernel_launches()  # kernels launched before the timed region (ncu -s)
        torch.cuda.synchronize()
        h0 = time.time()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx --nvtx-include timed/ selects the timed solves
        for k in range(args.steps):
            okk, stats = pb.solve(sp)
            ok &= okk
        torch.cuda.nvtx.range_pop()
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.time())
    launches = T.tmamg_kernel_launches() - launches0
    total_ms = max_over_ranks(t0.elapsed_time(t1), world)
    solves_per_s = whole_job_rate(nsys * args.steps, world, total_ms)
    # end to end through the public API with host buffers (page-locked): every step copies b in
    # and x out inside tmamg_solve
    bh_t = torch.from_numpy(pb.b.view(np.float64).copy()).pin_memory()
    xh_t = torch.zeros(nsys * V * 24, dtype=torch.float64).pin_memory()
    bh, xh = bh_t.numpy(), xh_t.numpy()
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_ok = True
    for k in range(args.steps):
        rc, st_ = T.tmamg_solve(pb.ctx, bh, pb.nrhs, pb.mus, len(pb.mus), xh, 0, sp)
        e2e_ok &= rc == 0
    e2e_s = max_over_ranks(time.perf_counter() - t, world)
    # per-kernel shares of one more (profiled) solve, and the fine stencil (the operator the metric
    # names) timed alone on the same context and systems
    rec, prof_ms, prof_stats = kernel_profile(pb, sp, stream)
    kernels = kernel_rooflines(pb, rec, prof_ms, prof_stats)
    kern_ms = measure_dirac(T, pb.ctx, nsys, np.array([pb.mus[n % len(pb.mus)] for n in range(nsys)]), 10, stream)
    hbm, _, peak_src = read_peaks()
    bytes_per_apply = dirac_bytes_per_site(nsys, 32) * V
    achieved = bytes_per_apply / (kern_ms * 1e-3) / 1e9
    fb32 = T.tmamg_bundle_bytes(pb.ctx, nsys, 32)
    fb64 = T.tmamg_bundle_bytes(pb.ctx, nsys, 64)
    m = wl["solve"]["restart"]
    vec_bytes = (2 * m + 1 + 3) * fb32 + 2 * fb64 + pb.nrhs * V * 12 * 16
    line = {
        "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f16+f64", "data": "synthetic",
        "config": {"workload": wl["name"], "lattice": "x".join(str(v) for v in pb.L), "systems_per_step": nsys,
                   "nrhs": pb.nrhs, "twisted_masses": pb.mus, "kappa": pb.kappa, "kappa_source": pb.ksrc,
                   "c_sw": wl["c_sw"], "tol": wl["solve"]["tol"], "amg": wl["amg"],
                   "precision": "FP32 fine stencil, SAP, transfers and inner FGMRES; FP16 coarse operators on the "
                                "tensor cores with FP32 accumulation; FP64 outer residuals",
                   "setup_seconds": pb.setup_seconds, "all_converged": bool(ok and e2e_ok),
                   "iterations": stats_summary(stats),
                   "solver_vector_bytes": int(vec_bytes),
                   "l2": "inputs larger than the 129 MB L2 (one FP32 bundle %.1f GB)" % (fb32 / 1e9)},
        "roofline": dominant_roofline(kernels),
        "dirac_op": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": kernel_traffic("dirac_f32", pb.L, nsys), "peak_source": peak_src,
                     "kernel": "dirac_kernel<float,2> (fine stencil, %d systems, timed alone)" % nsys,
                     "algorithmic_bytes_per_launch": bytes_per_apply, "launch_ms": kern_ms},
        "kernels": {"profiled_solve_ms": prof_ms, "by_kernel": kernels},
        "e2e": {"value": whole_job_rate(nsys * args.steps, world, e2e_s * 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": int(pb.b.nbytes), "d2h_bytes_per_step": int(nsys * V * 24 * 8)},
        "gpu_launches": int(launches),
        "launches_before_timed": int(launches0),
        "clocks": clk.result,
        "autotune": T.tmamg_autotune_report(),
    }
    pb.close()
    del bh_t, xh_t
    if args.variants:
        line["variants"] = run_variants(args, rank, stream)
    return line


def dominant_roofline(kernels):
    """The roofline entry of the kernel with the largest time share that has an algorithmic count."""
    best = None
    for name, e in kernels.items():
        if "achieved" in e and (best is None or e["share"] > kernels[best]["share"]):
            best = name
    if best is None:
        return None
    e = kernels[best]
    r = {k: e[k] for k in ("bound", "achieved", "peak", "unit", "frac", "peak_source")}
    r.update(kernel=best, share_of_solve=e["share"], launches_in_solve=e["launches"], launch_ms=e["ms_per_launch"],
             traffic=e.get("traffic"))
    for k in ("algorithmic_bytes_per_launch", "algorithmic_flops_per_launch"):
        if k in e:
            r[k] = e[k]
    return r


def run_variants(args, rank, stream):
    """Other workloads and other forms of the method, each timed with CUDA events; a variant that
    fails is recorded with its error and the headline line is still printed."""
    import torch
    from paper_2201_03872_gb300 import tmamg as T
    out = {}
    steps = max(1, min(args.steps, args.variant_steps))

    def guarded(label, fn):
        try:
            fn()
        except Exception as exc:  # noqa: BLE001
            out[label] = {"error": f"{type(exc).__name__}: {exc}"}

    def record(label, pb, ms, ok, stats, nrhs=None, **extra):
        nr = pb.nrhs if nrhs is None else nrhs
        n = nr * len(pb.mus)
        out[label] = dict({"workload": pb.wl["name"], "systems_per_step": n, "solves_per_s": n / (ms * 1e-3),
                           "ms_per_step": ms, "steps": steps, "all_converged": bool(ok),
                           "iterations": stats_summary(stats)}, **extra)

    def batched():
        pb = Problem(WORKLOADS["batched"], rank, stream)
        try:
            ms, ok, st_ = timed_solves(pb, pb.params(), steps, stream)
            record("batched_multishift_40_systems", pb, ms, ok, st_, setup_seconds=pb.setup_seconds)
            ms, ok, st_ = timed_solves(pb, pb.params(coarse_solver=1), steps, stream)
            record("batched_multishift_block_gmres_coarse", pb, ms, ok, st_)
        finally:
            pb.close()

    def precision():
        pb = Problem(WORKLOADS["precision"], rank, stream)
        try:
            ms, ok, st_ = timed_solves(pb, pb.params(), steps, stream)
            record("precision_form", pb, ms, ok, st_, setup_seconds=pb.setup_seconds)
            guarded("single_system", lambda: record("single_system", pb, *timed_solves(pb, pb.params(), steps,
                                                                                      stream, 1), nrhs=1))
            # the plain comparator: one system, every vector, operator and reduction in FP64
            guarded("plain_fp64_single_system", lambda: record(
                "plain_fp64_single_system", pb, *timed_solves(pb, pb.params(precision=64), steps, stream, 1), nrhs=1))
            guarded("block_gmres_coarse", lambda: record(
                "block_gmres_coarse", pb, *timed_solves(pb, pb.params(coarse_solver=1), steps, stream)))

            def learned():
                t = time.time()
                rep = T.tmamg_nn_train(pb.ctx, T.tmamg_default_nn_params(pairs=48, batch=12, epochs=30, lr=2e-3,
                                                                          mu=pb.mus[0], gate_systems=4))
                torch.cuda.synchronize()
                record("learned_step", pb, *timed_solves(pb, pb.params(use_nn=2), steps, stream),
                       train_seconds=time.time() - t, loss_first=rep.loss_first, loss_last=rep.loss_last,
                       gate_iterations_plain=rep.iters_plain, gate_iterations_with_step=rep.iters_nn,
                       gate_enabled=bool(rep.enabled))

            guarded("learned_step", learned)

            def doublet():
                # the non-degenerate doublet on the same lattice and setup: the 12 point sources as 6 flavour
                # pairs (u, d), twisted mass mu and splitting eps = 2/3 mu, one doublet solve per pair
                nd = pb.nrhs // 2
                eps = [2.0 * m / 3.0 for m in pb.mus]
                xd = torch.zeros(nd * len(pb.mus) * 2 * pb.V * 24, dtype=torch.float64, device="cuda")
                sp = pb.params()

                def solve_d():
                    rc, st = T.tmamg_solve_doublet(pb.ctx, pb.bd, nd, pb.mus, eps, len(pb.mus), xd, 1, sp)
                    ok = rc == 0 and all(q.status == 0 and q.true_rel_res <= pb.wl["solve"]["tol"] for q in st)
                    return ok, st

                solve_d()
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ok = True
                for _ in range(steps):
                    okk, st_ = solve_d()
                    ok &= okk
                z.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(z) / steps
                n = nd * len(pb.mus)
                out["doublet_6_pairs"] = {"workload": pb.wl["name"] + "; as 6 non-degenerate doublets, eps = 2/3 mu",
                                          "doublets_per_step": n, "doublet_solves_per_s": n / (ms * 1e-3),
                                          "flavour_fields_per_s": 2 * n / (ms * 1e-3), "ms_per_step": ms,
                                          "steps": steps, "all_converged": bool(ok),
                                          "iterations": stats_summary(st_)}
                del xd

            guarded("doublet_6_pairs", doublet)
        finally:
            pb.close()

        def three():
            pb3 = Problem(WORKLOADS["precision"], rank, stream,
                          dict(levels=3, agg2=(2, 2, 2, 2), nv2=32, setup_gmres_steps=20))
            try:
                sp = pb3.params(mid_tol=7e-2, mid_restart=10, mid_maxiter=50, mid_smooth=3)
                record("precision_form_three_level", pb3, *timed_solves(pb3, sp, steps, stream),
                       setup_seconds=pb3.setup_seconds)
            finally:
                pb3.close()

        guarded("precision_form_three_level", three)

    def largest_fp64():
        # the plain comparator on the headline lattice: one system, two levels (the FP64 solver's form),
        # every vector, operator and reduction in FP64; one timed solve
        wl = dict(WORKLOADS["largest"], nrhs=1, mus=[WORKLOADS["largest"]["mus"][0]],
                  setup=dict(WORKLOADS["largest"]["setup"], levels=2),
                  solve=dict(tol=1e-10, restart=10, max_outer=60, coarse_tol=0.1, coarse_restart=40,
                             coarse_maxiter=400))
        pb = Problem(wl, rank, stream)
        try:
            ms, ok, st_ = timed_solves(pb, pb.params(precision=64), 1, stream)
            record("largest_plain_fp64_single_system", pb, ms, ok, st_, setup_seconds=pb.setup_seconds, steps=1,
                   note="40^3x80, one Gaussian rhs at mu=0.0015, two-level FP64 AMG, FGMRES(10)")
        finally:
            pb.close()

    def learned_c4():
        # the learned step at its stated size: 4096 (residual, error) pairs from the plain solver on the same
        # field, collected and trained 16 batches of 8 at a time (a full set of pairs would not fit in HBM),
        # then the gate and the same solve with and without the step (opt-in: pair collection and training
        # take about 17 minutes on one GB300)
        pb = Problem(WORKLOADS["learned"], rank, stream)
        try:
            ms, ok, st_ = timed_solves(pb, pb.params(), steps, stream)
            record("learned_config4_plain", pb, ms, ok, st_, setup_seconds=pb.setup_seconds)
            t = time.time()
            rep = T.tmamg_nn_train(pb.ctx, T.tmamg_default_nn_params(pairs=4096, batch=8, window=16, epochs=2,
                                                                      lr=2e-3, pair_tol=1e-3, mu=pb.mus[0],
                                                                      gate_systems=8))
            torch.cuda.synchronize()
            train_s = time.time() - t
            record("learned_config4_with_step", pb, *timed_solves(pb, pb.params(use_nn=2), steps, stream),
                   train_seconds=train_s, pairs=4096, loss_first=rep.loss_first, loss_last=rep.loss_last,
                   gate_iterations_plain=rep.iters_plain, gate_iterations_with_step=rep.iters_nn,
                   gate_enabled=bool(rep.enabled))
        finally:
            pb.close()

    guarded("batched_multishift_40_systems", batched)
    guarded("precision_form", precision)
    guarded("largest_plain_fp64_single_system", largest_fp64)
    if args.learned_c4:
        guarded("learned_config4", learned_c4)
    return out


def cores_used(fn):
    """Run fn and return (result, wall seconds, threads it kept busy = process CPU time / wall time)."""
    c0, t0 = time.process_time(), time.perf_counter()
    r = fn()
    wall = time.perf_counter() - t0
    return r, wall, max(1, round((time.process_time() - c0) / max(wall, 1e-9)))


def oracle_amg_iteration(wl, Ls):
    """Closure timing one fine-level AMG iteration of the FP64 numpy oracle for one system on lattice Ls
    with the workload's gauge recipe: the FGMRES operator application, restriction and prolongation with a
    random P (Nv = 24, 4^4 aggregates), the residual and the SAP smoother with the workload's settings
    (4^4 blocks, the solve's cycles and MR steps)."""
    from oracle import dirac, sap as osap, amg
    kappa, _ = kappa_for(wl["L"], wl["eps"], wl["seed"])
    U = synth.gauge_field(Ls, wl["eps"], seed=wl["seed"])
    op = dirac.Operator(U, kappa, wl["c_sw"])
    x = synth.gaussian_spinors(Ls, 1, seed=7)[0]
    bop = osap.BlockOperator(op, (4, 4, 4, 4))
    Vt = synth.gaussian_spinors(Ls, 24, seed=8)
    P = amg.Prolongation(amg.FineLevel.to_chi(Vt), Ls, (4, 4, 4, 4))
    mu = wl["mus"][0]

    def it():
        y = op.apply(x, mu)
        rc = P.restrict(amg.FineLevel.to_chi(y))
        e = amg.FineLevel.to_spin(P.prolong(rc))
        r2 = y - op.apply(e, mu)
        return e + osap.sap(op, r2, mu, (4, 4, 4, 4),
                            cycles=wl["solve"].get("sap_cycles") or wl["setup"]["sap_cycles"],
                            mr_steps=wl["solve"].get("sap_mr_steps") or wl["setup"]["sap_mr_steps"], bop=bop)

    return it, op, x, mu


def sample_lattice(L):
    """The numpy oracle's bounded sample: the workload's own lattice up to 16^3 x 32 sites (one AMG
    iteration there takes the oracle about 12 s), else 16^3 x 32 with the same gauge recipe, the
    per-site cost being the same on any volume."""
    if int(np.prod(L)) > 16 ** 3 * 32:
        return (16, 16, 16, 32)
    return tuple(L)


def cpu_solve_baseline(wl, iters_per_solve, nsys, steps=0, warmup=0):
    """The FP64 numpy oracle as it stands, one system at a time: one fine-level AMG iteration on a
    bounded sample lattice, timed on the host, scaled by the volume ratio to the workload's lattice and
    multiplied by the GPU solver's FGMRES iteration count. Setup and coarse solves are left out, so this
    over-estimates the CPU rate. With steps > 0 (the reference arm) the iteration is expressed in oracle
    operator applications once, then warmup + steps applications are timed one by one."""
    Ls = sample_lattice(wl["L"])
    scale = float(np.prod(wl["L"])) / float(np.prod(Ls))
    it, op, x, mu = oracle_amg_iteration(wl, Ls)
    _, dt, cores = cores_used(it)
    lat = "x".join(str(v) for v in Ls)
    if steps <= 0:
        per_solve = dt * scale * iters_per_solve
        return {"value": 1.0 / per_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": f"numpy FP64 oracle, extrapolated: one fine-level AMG iteration for one system on {lat} "
                          f"({dt:.1f} s wall, about {cores} busy thread(s)) x volume ratio {scale:g} x "
                          f"{iters_per_solve} FGMRES iterations per solve; setup and coarse solves excluded"}
    t = time.perf_counter()
    op.apply(x, mu)
    per_iter = dt / (time.perf_counter() - t)
    times = []
    for k in range(warmup + steps):
        t = time.perf_counter()
        op.apply(x, mu)
        if k >= warmup:
            times.append(time.perf_counter() - t)
    t_op = float(np.mean(times))
    return {"value": 1.0 / (t_op * per_iter * scale * iters_per_solve), "unit": "solves/s", "cores": cores,
            "kind": "oracle",
            "sample": f"numpy FP64 oracle, extrapolated: {warmup} + {steps} timed operator applications on {lat} "
                      f"(mean {t_op:.2f} s) x {per_iter:.1f} applications per fine-level AMG iteration x volume "
                      f"ratio {scale:g} x {iters_per_solve} iterations per solve; about {cores} busy thread(s); "
                      f"setup and coarse solves excluded"}


def cpu_dirac_baseline(steps=0, warmup=0):
    """The FP64 oracle operator on the precision-form lattice (4 systems), timed on the host cores:
    about 8 s of applications, or (the reference arm) warmup + steps applications timed one by one."""
    from oracle import dirac
    wl = WORKLOADS["precision"]
    L = wl["L"]
    V = int(np.prod(L))
    kappa, _ = kappa_for(L, wl["eps"], wl["seed"])
    U = synth.gauge_field(L, wl["eps"], seed=wl["seed"])
    op = dirac.Operator(U, kappa, wl["c_sw"])
    nsys = 4
    x = synth.gaussian_spinors(L, nsys, seed=7)
    mu = np.full(nsys, wl["mus"][0])
    op.apply(x[:1], mu[:1])
    c0 = time.process_time()
    if steps > 0:
        times = []
        t_all = time.perf_counter()
        for k in range(warmup + steps):
            t = time.perf_counter()
            op.apply(x, mu)
            if k >= warmup:
                times.append(time.perf_counter() - t)
        dt, reps = float(np.mean(times)), steps
        wall = time.perf_counter() - t_all
    else:
        t = time.perf_counter()
        reps = 0
        while True:
            op.apply(x, mu)
            reps += 1
            if time.perf_counter() - t > 8.0:
                break
        wall = time.perf_counter() - t
        dt = wall / reps
    cores = max(1, round((time.process_time() - c0) / max(wall, 1e-9)))
    gbs = dirac_bytes_per_site(nsys, 32) * V / dt / 1e9
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"numpy FP64 oracle D(mu) on 16^3x32 with {nsys} systems, {reps} applications, about {cores} "
                      "busy thread(s); bytes counted with the same FP32 algorithmic formula as the GPU line"}


# FGMRES iterations per solve of the GPU solver on each workload (the CPU extrapolation of the
# reference arm uses them when it runs without a GPU measurement beside it)
ITERS_PER_SOLVE = {"largest": 15, "batched": 21, "precision": 16, "learned": 16}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--what", default="solve", choices=["solve", "dirac", "sap", "eo"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="solve: default the largest workload; dirac/sap: the lattice, default 16^3x32")
    ap.add_argument("--nsys", type=int, default=None,
                    help="dirac/sap diagnostic modes: systems per launch (default 12 for dirac, 16 for sap)")
    ap.add_argument("--variant-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the other workloads and forms of the method")
    ap.add_argument("--learned-c4", action="store_true",
                    help="add the learned step at 32^3x64 with 4096 training pairs to the variants (about 20 minutes)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.what == "solve" and args.workload is None:
        args.workload = HEADLINE
    world, rank, local = dist_init()
    if args.impl == "reference":
        if rank != 0:
            return
        wl = WORKLOADS[args.workload or "precision"]
        cb = (cpu_solve_baseline(wl, ITERS_PER_SOLVE[args.workload], wl["nrhs"] * len(wl["mus"]), steps=args.steps,
                                 warmup=args.warmup) if args.what == "solve"
              else cpu_dirac_baseline(steps=args.steps, warmup=args.warmup))
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": cb["unit"], "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": wl["name"] if args.what == "solve"
                           else dirac_workload(WORKLOADS["precision"]["L"], WORKLOADS["precision"]["nrhs"])},
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
    run = {"solve": run_solve, "dirac": run_dirac, "sap": run_sap, "eo": run_eo}[args.what]
    line = run(args, world, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1 and args.what in ("solve", "dirac"):
            wl = WORKLOADS[args.workload or "precision"]
            line["cpu_baseline"] = (cpu_solve_baseline(wl, line["config"]["iterations"]["fgmres"],
                                                       line["config"]["systems_per_step"])
                                    if args.what == "solve" else cpu_dirac_baseline())
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

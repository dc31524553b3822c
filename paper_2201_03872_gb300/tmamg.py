"""Thin ctypes binding of the tmamg C ABI (include/tmamg.h).

Argument marshalling only: every step of the method runs in the CUDA library
libtmamg.so. Functions keep the C names; they take plain Python numbers,
numpy arrays (host memory) or integer device pointers (e.g. torch's
``tensor.data_ptr()``), and raise TmamgError on a negative status.
There is no fallback: if the library is missing, loading fails loudly.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtmamg.so")

TMAMG_OK = 0
TMAMG_NOT_CONVERGED = 1
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_ARG", -2: "ERR_STATE", -3: "ERR_OOM", -4: "ERR_CUDA",
                -5: "ERR_NONFINITE", -6: "ERR_TIMEOUT"}


class TmamgError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class SetupParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("agg", (ctypes.c_int * 4) * 2), ("nv", ctypes.c_int * 2),
                ("sap_block", ctypes.c_int * 4), ("sap_cycles", ctypes.c_int), ("sap_mr_steps", ctypes.c_int),
                ("setup_iters", ctypes.c_int), ("mu_setup", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("setup_gmres_steps", ctypes.c_int)]


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("coarse_restart", ctypes.c_int), ("coarse_maxiter", ctypes.c_int),
                ("coarse_solver", ctypes.c_int), ("delta_mu", ctypes.c_double), ("precision", ctypes.c_int),
                ("use_nn", ctypes.c_int), ("poll", ctypes.c_int), ("coarse_precision", ctypes.c_int),
                ("mid_tol", ctypes.c_double), ("mid_restart", ctypes.c_int), ("mid_maxiter", ctypes.c_int),
                ("mid_smooth", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("sap_cycles", ctypes.c_int),
                ("sap_mr_steps", ctypes.c_int)]


class SystemStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("coarse_iters", ctypes.c_int), ("true_rel_res", ctypes.c_double)]


class NNParams(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("batch", ctypes.c_int), ("epochs", ctypes.c_int), ("lr", ctypes.c_double),
                ("pair_tol", ctypes.c_double), ("mu", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("gate_systems", ctypes.c_int), ("window", ctypes.c_int)]


class NNReport(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("iters_plain", ctypes.c_int),
                ("iters_nn", ctypes.c_int), ("enabled", ctypes.c_int)]


NN_WEIGHTS = 9 * (8 * 4 + 8 * 8 + 4 * 8)  # complex numbers in the three layers

_lib = None


def lib():
    """Load libtmamg.so (built by __graft_entry__.build() / paper_2201_03872_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtmamg.so not built ({LIB_PATH}); run python -m paper_2201_03872_gb300.build")
        _lib = ctypes.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double

# name -> (restype, argtypes); the list is checked against include/tmamg.h by the tests
SIGNATURES = {
    "tmamg_default_setup_params": (None, [ctypes.POINTER(SetupParams)]),
    "tmamg_default_solve_params": (None, [ctypes.POINTER(SolveParams)]),
    "tmamg_create": (I, [ctypes.POINTER(ctypes.c_int), I, P, ctypes.POINTER(P)]),
    "tmamg_destroy": (I, [P]),
    "tmamg_last_error": (ctypes.c_char_p, [P]),
    "tmamg_volume": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
    "tmamg_kernel_launches": (ctypes.c_uint64, []),
    "tmamg_load_gauge": (I, [P, P, I]),
    "tmamg_set_operator": (I, [P, D, D]),
    "tmamg_bundle_bytes": (ctypes.c_size_t, [P, I, I]),
    "tmamg_pack": (I, [P, P, P, I, I]),
    "tmamg_unpack": (I, [P, P, P, I, I]),
    "tmamg_dirac": (I, [P, P, P, I, P, I]),
    "tmamg_dirac_doublet": (I, [P, P, P, I, P, P, I]),
    "tmamg_dirac_eo": (I, [P, P, P, I, P, I]),
    "tmamg_apply": (I, [P, P, P, I, P, I]),
    "tmamg_setup": (I, [P, ctypes.POINTER(SetupParams), P]),
    "tmamg_setup_from_vectors": (I, [P, ctypes.POINTER(SetupParams), P]),
    "tmamg_solve": (I, [P, P, I, P, I, P, I, ctypes.POINTER(SolveParams), P]),
    "tmamg_solve_doublet": (I, [P, P, I, P, P, I, P, I, ctypes.POINTER(SolveParams), P]),
    "tmamg_coarse_bundle_bytes": (ctypes.c_size_t, [P, I, I]),
    "tmamg_sap": (I, [P, P, P, I, P, ctypes.POINTER(ctypes.c_int), I, I]),
    "tmamg_sap_noalloc": (I, [P, P, P, I, P, ctypes.POINTER(ctypes.c_int), I, I]),
    "tmamg_restrict": (I, [P, I, P, P, I]),
    "tmamg_prolong": (I, [P, I, P, P, I]),
    "tmamg_coarse_apply": (I, [P, I, P, P, I, P, I]),
    "tmamg_coarse_solve": (I, [P, I, P, P, I, P, I, ctypes.POINTER(SolveParams), ctypes.POINTER(ctypes.c_int)]),
    "tmamg_default_nn_params": (None, [ctypes.POINTER(NNParams)]),
    "tmamg_nn_init": (I, [P, ctypes.c_uint64]),
    "tmamg_nn_set_weights": (I, [P, P]),
    "tmamg_nn_get_weights": (I, [P, P]),
    "tmamg_nn_forward": (I, [P, P, P, I, I]),
    "tmamg_nn_loss_grad": (I, [P, P, P, I, ctypes.POINTER(ctypes.c_double), P]),
    "tmamg_nn_train": (I, [P, ctypes.POINTER(NNParams), ctypes.POINTER(NNReport)]),
    "tmamg_debug_bounded_wait": (I, [ctypes.c_longlong, I]),
    "tmamg_profile_enable": (I, [I]),
    "tmamg_autotune": (I, [I]),
    "tmamg_autotune_force": (I, [I]),
    "tmamg_autotune_report": (I, [ctypes.c_char_p, ctypes.c_size_t]),
    "tmamg_profile_report": (I, [ctypes.c_char_p, ctypes.c_size_t]),
}


def _declare(L):
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(x):
    """Host numpy array -> its address; int -> as is (a device pointer); torch tensor -> data_ptr()."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check(name, ctx, rc):
    if rc < 0:
        msg = lib().tmamg_last_error(ctx).decode() if ctx else ""
        raise TmamgError(name, rc, msg)
    return rc


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def tmamg_default_setup_params():
    p = SetupParams()
    lib().tmamg_default_setup_params(ctypes.byref(p))
    return p


def tmamg_default_solve_params():
    p = SolveParams()
    lib().tmamg_default_solve_params(ctypes.byref(p))
    return p


def tmamg_create(L, bc_t=-1, stream=0):
    arr = (ctypes.c_int * 4)(*[int(v) for v in L])
    out = P()
    rc = lib().tmamg_create(arr, int(bc_t), P(stream or None), ctypes.byref(out))
    if rc < 0:
        raise TmamgError("tmamg_create", rc, "invalid lattice/bc or device allocation failed")
    return out.value


def tmamg_destroy(ctx):
    return lib().tmamg_destroy(ctx)


def tmamg_last_error(ctx):
    return lib().tmamg_last_error(ctx).decode()


def tmamg_volume(ctx):
    v = ctypes.c_int64()
    _check("tmamg_volume", ctx, lib().tmamg_volume(ctx, ctypes.byref(v)))
    return v.value


def tmamg_kernel_launches():
    return lib().tmamg_kernel_launches()


def tmamg_load_gauge(ctx, U, on_device=None):
    """U: complex128 numpy array [Lt, Lz, Ly, Lx, 4, 3, 3] (host) or a device pointer / tensor."""
    if isinstance(U, np.ndarray):
        U = np.ascontiguousarray(U.astype(np.complex128))
        return _check("tmamg_load_gauge", ctx, lib().tmamg_load_gauge(ctx, _ptr(U), 0))
    return _check("tmamg_load_gauge", ctx, lib().tmamg_load_gauge(ctx, _ptr(U), 1 if on_device is None else on_device))


def tmamg_set_operator(ctx, kappa, c_sw):
    return _check("tmamg_set_operator", ctx, lib().tmamg_set_operator(ctx, float(kappa), float(c_sw)))


def tmamg_bundle_bytes(ctx, nsys, prec):
    return lib().tmamg_bundle_bytes(ctx, int(nsys), int(prec))


def tmamg_pack(ctx, x_field, x_bundle, nsys, prec):
    return _check("tmamg_pack", ctx, lib().tmamg_pack(ctx, _ptr(x_field), _ptr(x_bundle), int(nsys), int(prec)))


def tmamg_unpack(ctx, x_bundle, x_field, nsys, prec):
    return _check("tmamg_unpack", ctx, lib().tmamg_unpack(ctx, _ptr(x_bundle), _ptr(x_field), int(nsys), int(prec)))


def tmamg_dirac(ctx, x_bundle, y_bundle, nsys, mu, prec):
    m = _f64(mu)
    return _check("tmamg_dirac", ctx, lib().tmamg_dirac(ctx, _ptr(x_bundle), _ptr(y_bundle), int(nsys), _ptr(m),
                                                        int(prec)))


def tmamg_dirac_doublet(ctx, x_bundle, y_bundle, npair, mu, eps, prec):
    m = _f64(mu)
    e = _f64(eps)
    return _check("tmamg_dirac_doublet", ctx,
                  lib().tmamg_dirac_doublet(ctx, _ptr(x_bundle), _ptr(y_bundle), int(npair), _ptr(m), _ptr(e),
                                            int(prec)))


def tmamg_dirac_eo(ctx, x_bundle, y_bundle, nsys, mu, prec):
    m = _f64(mu)
    return _check("tmamg_dirac_eo", ctx, lib().tmamg_dirac_eo(ctx, _ptr(x_bundle), _ptr(y_bundle), int(nsys), _ptr(m),
                                                              int(prec)))


def tmamg_apply(ctx, x_field, y_field, nsys, mu, prec):
    m = _f64(mu)
    return _check("tmamg_apply", ctx, lib().tmamg_apply(ctx, _ptr(x_field), _ptr(y_field), int(nsys), _ptr(m),
                                                        int(prec)))


def setup_params(levels=2, agg=(4, 4, 4, 4), nv=24, sap_block=(4, 4, 4, 4), sap_cycles=2, sap_mr_steps=3,
                 setup_iters=5, mu_setup=0.0, seed=1, agg2=(2, 2, 2, 2), nv2=32, setup_gmres_steps=20):
    p = tmamg_default_setup_params()
    p.levels = levels
    for d in range(4):
        p.agg[0][d] = agg[d]
        p.agg[1][d] = agg2[d]
        p.sap_block[d] = sap_block[d]
    p.nv[0] = nv
    p.nv[1] = nv2
    p.sap_cycles = sap_cycles
    p.sap_mr_steps = sap_mr_steps
    p.setup_iters = setup_iters
    p.mu_setup = mu_setup
    p.seed = seed
    p.setup_gmres_steps = setup_gmres_steps
    return p


def solve_params(**kw):
    p = tmamg_default_solve_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tmamg_setup(ctx, params, start_vectors=None):
    return _check("tmamg_setup", ctx, lib().tmamg_setup(ctx, ctypes.byref(params), _ptr(start_vectors)))


def tmamg_setup_from_vectors(ctx, params, test_vectors):
    return _check("tmamg_setup_from_vectors", ctx,
                  lib().tmamg_setup_from_vectors(ctx, ctypes.byref(params), _ptr(test_vectors)))


def tmamg_solve(ctx, b, nrhs, mu, nshift, x, on_device, params=None):
    """Returns (status, stats) with stats a list of SystemStats; raises on a negative status."""
    m = _f64(mu)
    stats = (SystemStats * (nrhs * nshift))()
    pp = ctypes.byref(params) if params is not None else None
    rc = lib().tmamg_solve(ctx, _ptr(b), int(nrhs), _ptr(m), int(nshift), _ptr(x), int(on_device), pp,
                           ctypes.cast(stats, P))
    _check("tmamg_solve", ctx, rc)
    return rc, list(stats)


def tmamg_solve_doublet(ctx, b, nrhs, mu, eps, nshift, x, on_device, params=None):
    """Returns (status, stats), one SystemStats per doublet (rhs, shift); raises on a negative status."""
    m = _f64(mu)
    e = _f64(eps)
    stats = (SystemStats * (nrhs * nshift))()
    pp = ctypes.byref(params) if params is not None else None
    rc = lib().tmamg_solve_doublet(ctx, _ptr(b), int(nrhs), _ptr(m), _ptr(e), int(nshift), _ptr(x), int(on_device),
                                   pp, ctypes.cast(stats, P))
    _check("tmamg_solve_doublet", ctx, rc)
    return rc, list(stats)


def tmamg_coarse_bundle_bytes(ctx, level, nsys):
    return lib().tmamg_coarse_bundle_bytes(ctx, int(level), int(nsys))


def tmamg_sap(ctx, r_bundle, e_bundle, nsys, mu, block, cycles, mr_steps):
    m = _f64(mu)
    blk = (ctypes.c_int * 4)(*[int(v) for v in block])
    return _check("tmamg_sap", ctx, lib().tmamg_sap(ctx, _ptr(r_bundle), _ptr(e_bundle), int(nsys), _ptr(m), blk,
                                                    int(cycles), int(mr_steps)))


def tmamg_sap_noalloc(ctx, r_bundle, e_bundle, nsys, mu, block, cycles, mr_steps):
    """tmamg_sap without device allocation (fixed-size library-held scratch; see the header)."""
    m = _f64(mu)
    blk = (ctypes.c_int * 4)(*[int(v) for v in block])
    return _check("tmamg_sap_noalloc", ctx, lib().tmamg_sap_noalloc(ctx, _ptr(r_bundle), _ptr(e_bundle), int(nsys),
                                                                    _ptr(m), blk, int(cycles), int(mr_steps)))


def tmamg_restrict(ctx, level, fine_bundle, coarse_bundle, nsys):
    return _check("tmamg_restrict", ctx, lib().tmamg_restrict(ctx, int(level), _ptr(fine_bundle),
                                                              _ptr(coarse_bundle), int(nsys)))


def tmamg_prolong(ctx, level, coarse_bundle, fine_bundle, nsys):
    return _check("tmamg_prolong", ctx, lib().tmamg_prolong(ctx, int(level), _ptr(coarse_bundle),
                                                            _ptr(fine_bundle), int(nsys)))


def tmamg_coarse_apply(ctx, level, x_bundle, y_bundle, nsys, mu, precision=16):
    m = _f64(mu)
    return _check("tmamg_coarse_apply", ctx, lib().tmamg_coarse_apply(ctx, int(level), _ptr(x_bundle),
                                                                      _ptr(y_bundle), int(nsys), _ptr(m),
                                                                      int(precision)))


def tmamg_coarse_solve(ctx, level, rc_bundle, xc_bundle, nrhs, mu, nshift, params):
    """Returns the number of coarse iterations taken."""
    m = _f64(mu)
    it = ctypes.c_int(0)
    _check("tmamg_coarse_solve", ctx, lib().tmamg_coarse_solve(ctx, int(level), _ptr(rc_bundle), _ptr(xc_bundle),
                                                                int(nrhs), _ptr(m), int(nshift), ctypes.byref(params),
                                                                ctypes.byref(it)))
    return it.value


def tmamg_autotune(on):
    """Launch-shape autotuning on (default) or off (process-wide); clears the recorded choices."""
    return lib().tmamg_autotune(int(bool(on)))


def tmamg_autotune_force(variant):
    return lib().tmamg_autotune_force(int(variant))


def tmamg_autotune_report():
    """{family/device/key: {"choice": v, "ms": [...]}} of the tuned launch shapes."""
    import json
    n = 1 << 16
    buf = ctypes.create_string_buffer(n)
    rc = lib().tmamg_autotune_report(buf, n)
    if rc < 0:
        raise TmamgError("tmamg_autotune_report", rc, "record longer than the buffer")
    return json.loads(buf.value.decode())


def tmamg_profile_enable(on):
    """Per-kernel CUDA-event timing of the library's launches (process-wide); clears the record."""
    return lib().tmamg_profile_enable(int(bool(on)))


def tmamg_profile_report():
    """{kernel: (launches, total_ms)} of the launches recorded since tmamg_profile_enable."""
    import json
    n = 1 << 16
    buf = ctypes.create_string_buffer(n)
    rc = lib().tmamg_profile_report(buf, n)
    if rc < 0:
        raise TmamgError("tmamg_profile_report", rc, "record longer than the buffer")
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


def tmamg_debug_bounded_wait(limit_cycles, unreachable_next):
    """Process-wide bound of the persistent coarse solver's barrier waits, and a one-shot
    unreachable barrier for the next persistent coarse solve (tests of the timeout path)."""
    return _check("tmamg_debug_bounded_wait", None, lib().tmamg_debug_bounded_wait(int(limit_cycles),
                                                                                  int(unreachable_next)))


def tmamg_default_nn_params(**kw):
    p = NNParams()
    lib().tmamg_default_nn_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tmamg_nn_init(ctx, seed=7):
    return _check("tmamg_nn_init", ctx, lib().tmamg_nn_init(ctx, int(seed)))


def tmamg_nn_set_weights(ctx, Ws):
    """Ws: the three complex weight arrays [9][cout][cin] (concatenated in order)."""
    flat = np.ascontiguousarray(np.concatenate([np.asarray(w, dtype=np.complex128).ravel() for w in Ws]))
    assert flat.size == NN_WEIGHTS
    return _check("tmamg_nn_set_weights", ctx, lib().tmamg_nn_set_weights(ctx, _ptr(flat)))


def tmamg_nn_get_weights(ctx):
    flat = np.zeros(NN_WEIGHTS, dtype=np.complex128)
    _check("tmamg_nn_get_weights", ctx, lib().tmamg_nn_get_weights(ctx, _ptr(flat)))
    return flat


def tmamg_nn_forward(ctx, r_bundle, y_bundle, nsys, bf16=False):
    return _check("tmamg_nn_forward", ctx, lib().tmamg_nn_forward(ctx, _ptr(r_bundle), _ptr(y_bundle), int(nsys),
                                                                  1 if bf16 else 0))


def tmamg_nn_loss_grad(ctx, r_bundle, e_bundle, nsys):
    loss = ctypes.c_double(0)
    grad = np.zeros(NN_WEIGHTS, dtype=np.complex128)
    _check("tmamg_nn_loss_grad", ctx, lib().tmamg_nn_loss_grad(ctx, _ptr(r_bundle), _ptr(e_bundle), int(nsys),
                                                               ctypes.byref(loss), _ptr(grad)))
    return loss.value, grad


def tmamg_nn_train(ctx, params):
    rep = NNReport()
    _check("tmamg_nn_train", ctx, lib().tmamg_nn_train(ctx, ctypes.byref(params), ctypes.byref(rep)))
    return rep

"""Thin Python binding of the C ABI in include/amg_gnn.h (argument marshalling only).

Every function here has the name of the C entry point it calls; every step of
the solve and of the network runs in libamggnn.so's CUDA kernels.  The
library must have been built (``__graft_entry__.build()``); importing this
module without it raises immediately -- there is no fallback.

Matrices are passed as any object with ``n_rows, n_cols, row_ptr, col, val``
(e.g. ``workloads.CSR``).  Device vectors are torch CUDA tensors (float64);
streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

AMG_OK = 0
AMG_ERR_ARG = -1
AMG_ERR_CUDA = -2
AMG_ERR_NOT_SPD = -3
AMG_ERR_DIVERGED = -4
AMG_ERR_STAGNATED = -5
AMG_ERR_MAXITER = -6
AMG_ERR_DEVICE_FLAG = -7
AMG_ERR_STATE = -8
AMG_FP64 = 0
AMG_FP32_IN_FP64 = 1
AMG_SMOOTHER_JACOBI = 0
AMG_SMOOTHER_GNN = 1
AMG_SMOOTHER_CHEB = 2
AMG_OUTER_REFINE = 0
AMG_OUTER_PCG = 1
AMG_GNN_FP32 = 0
AMG_GNN_BF16 = 1
AMG_SPLIT_SECOND_PASS = 1     # amg_setup_device: then the round-parallel second pass
AMG_SPLIT_RS_BLOCKS = 2       # amg_setup_device: block-local RS first pass instead of PMIS
AMG_GCIN_NUM_PARAMS = 55045        # GCIN width 64 (App. A.1)
AMG_GCIN_NUM_PARAMS_H32 = 37189    # GCIN width 32 (App. B.3)

SOLVE_STATUSES = (AMG_OK, AMG_ERR_DIVERGED, AMG_ERR_STAGNATED, AMG_ERR_MAXITER)


class AmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class amg_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_cols", C.c_int), ("nnz", C.c_longlong),
                ("row_ptr", C.POINTER(C.c_int)), ("col", C.POINTER(C.c_int)), ("val", C.POINTER(C.c_double))]


class amg_options(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("max_levels", C.c_int), ("max_coarse", C.c_int),
                ("max_iter", C.c_int), ("precision", C.c_int), ("smoother", C.c_int), ("omega", C.c_double),
                ("theta", C.c_double), ("device", C.c_int), ("gnn_precision", C.c_int),
                ("outer", C.c_int), ("fused_sweeps", C.c_int)]


_LIB = None


def lib():
    """The loaded libamggnn.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: build it with __graft_entry__.build() "
                               "(the solver has no CPU fallback)")
        _LIB = C.CDLL(_build.LIB)
        _declare(_LIB)
    return _LIB


def _declare(L):
    P, I, D, LL, V = C.c_void_p, C.c_int, C.c_double, C.c_longlong, None
    pd, pi, pf = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)
    sig = {
        "amg_default_options": (V, [C.POINTER(amg_options)]),
        "amg_create": (I, [C.POINTER(P), C.POINTER(amg_options)]),
        "amg_destroy": (V, [P]),
        "amg_last_error": (C.c_char_p, [P]),
        "amg_setup": (I, [P, C.POINTER(amg_csr)]),
        "amg_setup_device": (I, [P, C.POINTER(amg_csr), C.c_ulonglong, I]),
        "amg_load_hierarchy": (I, [P, I, C.POINTER(amg_csr), C.POINTER(amg_csr), C.POINTER(amg_csr)]),
        "amg_num_levels": (I, [P]),
        "amg_level_info": (I, [P, I, pi, C.POINTER(LL), C.POINTER(LL)]),
        "amg_get_level": (I, [P, I, pi, pi, pd, pi, pi, pd]),
        "amg_get_scales": (I, [P, pd]),
        "amg_set_jacobi": (I, [P, D]),
        "amg_set_coeffs": (I, [P, pd, I]),
        "amg_set_node_coeffs": (I, [P, pd, C.c_longlong]),
        "amg_get_smoother": (I, [P, I, pd]),
        "gnn_load_params": (I, [P, pf, LL]),
        "gnn_predict_coeffs": (I, [P, pd]),
        "amg_solve": (I, [P, pd, pd, D, pi, pd]),
        "amg_solve_device": (I, [P, P, P, D, P, pi, pd]),
        "amg_vcycle_device": (I, [P, P, P, P]),
        "amg_smooth_device": (I, [P, I, P, P, I, P]),
        "amg_spmv_device": (I, [P, I, P, P, P]),
        "amg_judge": (I, [P, pd, I, pd]),
        "amg_reroute": (I, [P, pd, I, pd, pi]),
        "amg_last_solve_rerouted": (I, [P]),
        "gcin_trainer_create": (I, [C.POINTER(P), I, I, pf, C.c_longlong]),
        "gcin_trainer_destroy": (V, [P]),
        "gcin_trainer_last_error": (C.c_char_p, [P]),
        "gcin_trainer_get_params": (I, [P, pf]),
        "gcin_trainer_set_params": (I, [P, pf, C.c_longlong]),
        "gcin_trainer_forward": (I, [P, I, C.POINTER(P), pd]),
        "gcin_trainer_backward": (I, [P, pd, pd]),
        "gcin_trainer_adam_step": (I, [P, D, D]),
        "amg_loss_grad": (I, [P, pd, pd, I, pd, pd]),
        "amg_kernel_launch": (I, [P, I, I, I, P, pd]),
        "gcin_tc_selftest": (I, [I, I, pf, pf, pf, pf, pf, C.POINTER(C.c_int)]),
        "amg_set_chebyshev": (I, [P, I]),
        "amg_get_chebyshev": (I, [P, I, pd, pd, pd]),
        "amg_vcycle_bytes": (I, [P, pd]),
        "amg_launch_count": (LL, []),
        "amg_residual_norm_noalloc": (I, [I, LL, P, P, P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(L, name):
            continue
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def exported_symbols():
    """Names of the C entry points this binding knows about."""
    return ["amg_default_options", "amg_create", "amg_destroy", "amg_last_error", "amg_setup", "amg_setup_device",
            "amg_load_hierarchy", "amg_num_levels", "amg_level_info", "amg_get_level", "amg_get_scales",
            "amg_set_jacobi", "amg_set_coeffs", "amg_set_node_coeffs", "amg_get_smoother", "gnn_load_params", "gnn_predict_coeffs",
            "amg_solve", "amg_solve_device", "amg_vcycle_device", "amg_smooth_device", "amg_spmv_device",
            "amg_judge", "amg_reroute", "amg_last_solve_rerouted", "gcin_trainer_create", "gcin_trainer_destroy", "gcin_trainer_last_error",
            "gcin_trainer_get_params", "gcin_trainer_set_params", "gcin_trainer_forward", "gcin_trainer_backward",
            "gcin_trainer_adam_step", "amg_loss_grad", "amg_kernel_launch", "amg_vcycle_bytes",
            "amg_launch_count", "amg_residual_norm_noalloc", "amg_set_chebyshev", "amg_get_chebyshev", "gcin_tc_selftest"]


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _csr(M, keep):
    rp = np.ascontiguousarray(M.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(M.col, dtype=np.int32)
    val = np.ascontiguousarray(M.val, dtype=np.float64)
    keep.extend([rp, col, val])
    return amg_csr(int(M.n_rows), int(M.n_cols), int(rp[-1]), _iptr(rp), _iptr(col), _dptr(val))


def _check(ctx, rc, allowed=(AMG_OK,)):
    if rc not in allowed:
        raise AmgError(rc, amg_last_error(ctx))
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _dev(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def amg_default_options(**overrides) -> amg_options:
    o = amg_options()
    lib().amg_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def amg_create(opt: amg_options | None = None, **overrides):
    if opt is None:
        opt = amg_default_options(**overrides)
    h = C.c_void_p()
    rc = lib().amg_create(C.byref(h), C.byref(opt))
    if rc != AMG_OK:
        raise AmgError(rc, amg_last_error(None))
    return h


def amg_destroy(ctx):
    lib().amg_destroy(ctx)


def amg_last_error(ctx) -> str:
    return lib().amg_last_error(ctx).decode()


def amg_setup(ctx, A):
    keep = []
    m = _csr(A, keep)
    return _check(ctx, lib().amg_setup(ctx, C.byref(m)))


def amg_setup_device(ctx, A, seed=0, split=AMG_SPLIT_SECOND_PASS):
    """split: AMG_SPLIT_* flags (0 = PMIS alone; True / False keep their
    former second-pass meaning)."""
    keep = []
    m = _csr(A, keep)
    return _check(ctx, lib().amg_setup_device(ctx, C.byref(m), int(seed) & 0xFFFFFFFFFFFFFFFF, int(split)))


def amg_load_hierarchy(ctx, A_list, P_list, R_list=None):
    keep = []
    nl = len(A_list)
    As = (amg_csr * nl)(*[_csr(A, keep) for A in A_list])
    Ps = (amg_csr * max(1, nl - 1))(*[_csr(P, keep) for P in P_list]) if nl > 1 else None
    Rs = (amg_csr * max(1, nl - 1))(*[_csr(R, keep) for R in R_list]) if (R_list and nl > 1) else None
    return _check(ctx, lib().amg_load_hierarchy(ctx, nl, As, Ps, Rs))


def amg_num_levels(ctx) -> int:
    return lib().amg_num_levels(ctx)


def amg_level_info(ctx, level):
    n, na, npp = C.c_int(), C.c_longlong(), C.c_longlong()
    _check(ctx, lib().amg_level_info(ctx, level, C.byref(n), C.byref(na), C.byref(npp)))
    return n.value, na.value, npp.value


def amg_get_level(ctx, level):
    """Returns (A, P) as dicts of numpy arrays (P is None on the coarsest level)."""
    n, na, npp = amg_level_info(ctx, level)
    arp, acol, aval = np.zeros(n + 1, np.int32), np.zeros(na, np.int32), np.zeros(na)
    coarse = level == amg_num_levels(ctx) - 1
    if coarse:
        _check(ctx, lib().amg_get_level(ctx, level, _iptr(arp), _iptr(acol), _dptr(aval), None, None, None))
        return dict(row_ptr=arp, col=acol, val=aval, n=n), None
    prp, pcol, pval = np.zeros(n + 1, np.int32), np.zeros(npp, np.int32), np.zeros(npp)
    _check(ctx, lib().amg_get_level(ctx, level, _iptr(arp), _iptr(acol), _dptr(aval), _iptr(prp), _iptr(pcol),
                                    _dptr(pval)))
    nc = amg_level_info(ctx, level + 1)[0]
    return dict(row_ptr=arp, col=acol, val=aval, n=n), dict(row_ptr=prp, col=pcol, val=pval, n=n, nc=nc)


def amg_get_scales(ctx) -> np.ndarray:
    s = np.zeros(amg_num_levels(ctx))
    _check(ctx, lib().amg_get_scales(ctx, _dptr(s)))
    return s


def amg_set_jacobi(ctx, omega=2.0 / 3.0):
    return _check(ctx, lib().amg_set_jacobi(ctx, float(omega)))


def amg_set_coeffs(ctx, c):
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, 5))
    return _check(ctx, lib().amg_set_coeffs(ctx, _dptr(c), c.shape[0]))


def amg_set_node_coeffs(ctx, c_levels):
    """c_levels[l]: (n_l x 5) per-node coefficients of smoothed level l."""
    flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1) for c in c_levels]))
    return _check(ctx, lib().amg_set_node_coeffs(ctx, _dptr(flat), flat.size))


def amg_get_smoother(ctx, level) -> np.ndarray:
    q = np.zeros(amg_level_info(ctx, level)[1])
    _check(ctx, lib().amg_get_smoother(ctx, level, _dptr(q)))
    return q


def gnn_load_params(ctx, theta):
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
    return _check(ctx, lib().gnn_load_params(ctx, _fptr(t), t.size))


def gnn_predict_coeffs(ctx) -> np.ndarray:
    c = np.zeros((amg_num_levels(ctx), 5))
    _check(ctx, lib().gnn_predict_coeffs(ctx, _dptr(c)))
    return c


def amg_solve(ctx, b, x0=None, rtol=1e-8, max_iter=None):
    """Returns (status, x, history)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    cap = (max_iter if max_iter is not None else 100000) + 1
    hist = np.zeros(cap)
    nvc = C.c_int()
    rc = _check(ctx, lib().amg_solve(ctx, _dptr(b), _dptr(x), float(rtol), C.byref(nvc), _dptr(hist)),
                SOLVE_STATUSES)
    return rc, x, hist[:nvc.value + 1].copy()


def amg_solve_device(ctx, d_b, d_x, rtol=1e-8, stream=None, hist_cap=100001):
    """Solve in place on device tensors; returns (status, history)."""
    hist = np.zeros(hist_cap)
    nvc = C.c_int()
    rc = _check(ctx, lib().amg_solve_device(ctx, _dev(d_b), _dev(d_x), float(rtol), _stream(stream),
                                            C.byref(nvc), _dptr(hist)), SOLVE_STATUSES)
    return rc, hist[:nvc.value + 1].copy()


def amg_vcycle_device(ctx, d_r, d_e, stream=None):
    return _check(ctx, lib().amg_vcycle_device(ctx, _dev(d_r), _dev(d_e), _stream(stream)))


def amg_smooth_device(ctx, level, d_b, d_u, n_sweeps, stream=None):
    return _check(ctx, lib().amg_smooth_device(ctx, level, _dev(d_b), _dev(d_u), int(n_sweeps), _stream(stream)))


def amg_spmv_device(ctx, level, d_x, d_y, stream=None):
    return _check(ctx, lib().amg_spmv_device(ctx, level, _dev(d_x), _dev(d_y), _stream(stream)))


def amg_judge(ctx, b, n_cycles=1) -> float:
    b = np.ascontiguousarray(b, dtype=np.float64)
    m = C.c_double()
    _check(ctx, lib().amg_judge(ctx, _dptr(b), int(n_cycles), C.byref(m)))
    return m.value


def amg_reroute(ctx, b, n_cycles=30):
    """(metric, smoother in use afterwards)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    m, sm = C.c_double(), C.c_int()
    _check(ctx, lib().amg_reroute(ctx, _dptr(b), int(n_cycles), C.byref(m), C.byref(sm)))
    return m.value, sm.value


def amg_last_solve_rerouted(ctx) -> bool:
    return bool(lib().amg_last_solve_rerouted(ctx))


def amg_loss_grad(ctx, c, f, n_vc=1):
    """(loss, dL/dc) of n_vc V-cycles from zero (Sec. 3.3)."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1, 5))
    f = np.ascontiguousarray(f, dtype=np.float64)
    loss = C.c_double()
    dc = np.zeros_like(c)
    _check(ctx, lib().amg_loss_grad(ctx, _dptr(c), _dptr(f), int(n_vc), C.byref(loss), _dptr(dc)))
    return loss.value, dc


(AMG_K_RESIDUAL, AMG_K_PINV, AMG_K_JACOBI, AMG_K_RESTRICT, AMG_K_PROLONG, AMG_K_OUTER, AMG_K_VCYCLE, AMG_K_MASWEEP,
 AMG_K_WF_PRE, AMG_K_WF_POST, AMG_K_EMPTY) = range(11)


def gcin_tc_selftest(x, W, bias, no_commit=False, device=0):
    """(y, h, flag) of one tensor-core GCIN layer on an identity graph."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    W = np.ascontiguousarray(W, dtype=np.float32)
    bias = np.ascontiguousarray(bias, dtype=np.float32)
    assert x.shape == (128, 64) and W.shape == (64, 64) and bias.shape == (64,)
    y = np.zeros((128, 64), dtype=np.float32)
    h = np.zeros((128, 64), dtype=np.float32)
    flag = C.c_int(-1)
    rc = lib().gcin_tc_selftest(int(device), 1 if no_commit else 0, _fptr(x), _fptr(W), _fptr(bias), _fptr(y),
                                _fptr(h), C.byref(flag))
    if rc != AMG_OK:
        raise AmgError(rc, "gcin_tc_selftest failed")
    return y, h, flag.value


def amg_set_chebyshev(ctx, degree=3):
    return _check(ctx, lib().amg_set_chebyshev(ctx, int(degree)))


def amg_get_chebyshev(ctx, level):
    """(rho, theta, delta) of the Chebyshev interval on `level`."""
    r, t, d = C.c_double(), C.c_double(), C.c_double()
    _check(ctx, lib().amg_get_chebyshev(ctx, int(level), C.byref(r), C.byref(t), C.byref(d)))
    return r.value, t.value, d.value


def amg_kernel_launch(ctx, kernel, level, reps, stream=None) -> float:
    """Enqueue `reps` launches of one kernel; returns algorithmic bytes per launch."""
    b = C.c_double()
    _check(ctx, lib().amg_kernel_launch(ctx, int(kernel), int(level), int(reps), _stream(stream), C.byref(b)))
    return b.value


def amg_vcycle_bytes(ctx) -> float:
    b = C.c_double()
    _check(ctx, lib().amg_vcycle_bytes(ctx, C.byref(b)))
    return b.value


def amg_launch_count() -> int:
    return int(lib().amg_launch_count())


def amg_residual_norm_noalloc(d_row_ptr, d_col, d_val, d_b, d_x, d_out, d_r=None, stream=None):
    """||b - A x|| and ||b|| into d_out[0:2] with no allocation; all arguments are device tensors.

    Every tensor must live on the current CUDA device (the library launches
    there and looks up its scratch array there); lengths are checked against
    n = d_b.numel() and nnz = d_col.numel() before the call, because a short
    buffer would become an out-of-bounds device access."""
    import torch
    n = d_b.numel()
    nnz = d_col.numel()
    for t, dt in ((d_row_ptr, torch.int32), (d_col, torch.int32)):
        assert t.is_cuda and t.dtype == dt and t.is_contiguous()
    dev = torch.cuda.current_device()
    tensors = [d_row_ptr, d_col, d_val, d_b, d_x, d_out] + ([d_r] if d_r is not None else [])
    if any(t.device.index != dev for t in tensors):
        raise ValueError("amg_residual_norm_noalloc: every tensor must be on the current CUDA device")
    if d_row_ptr.numel() != n + 1 or d_val.numel() != nnz or d_x.numel() != n or d_out.numel() < 2 or \
            (d_r is not None and d_r.numel() != n):
        raise ValueError("amg_residual_norm_noalloc: row_ptr needs n + 1 entries, val nnz, x and r n, out 2")
    rp = C.c_void_p(d_row_ptr.data_ptr())
    col = C.c_void_p(d_col.data_ptr())
    r = _dev(d_r) if d_r is not None else None
    rc = lib().amg_residual_norm_noalloc(n, nnz, rp, col, _dev(d_val), _dev(d_b), _dev(d_x), r, _dev(d_out),
                                         _stream(stream))
    if rc != AMG_OK:
        raise AmgError(rc, amg_last_error(None))
    return rc


# trainer --------------------------------------------------------------------
def _tcheck(tr, rc):
    if rc != AMG_OK:
        raise AmgError(rc, gcin_trainer_last_error(tr))
    return rc


def gcin_trainer_create(theta0, device=0, precision=AMG_GNN_BF16):
    t = np.ascontiguousarray(np.asarray(theta0, dtype=np.float32))
    if t.size not in (AMG_GCIN_NUM_PARAMS, AMG_GCIN_NUM_PARAMS_H32):
        raise ValueError("theta0 must have 55045 (width 64) or 37189 (width 32) entries")
    h = C.c_void_p()
    rc = lib().gcin_trainer_create(C.byref(h), int(device), int(precision), _fptr(t), t.size)
    if rc != AMG_OK:
        raise AmgError(rc, "gcin_trainer_create failed")
    h.n_params = t.size
    return h


def gcin_trainer_destroy(tr):
    lib().gcin_trainer_destroy(tr)


def gcin_trainer_last_error(tr) -> str:
    return lib().gcin_trainer_last_error(tr).decode()


def gcin_trainer_get_params(tr) -> np.ndarray:
    t = np.zeros(tr.n_params, np.float32)
    _tcheck(tr, lib().gcin_trainer_get_params(tr, _fptr(t)))
    return t


def gcin_trainer_set_params(tr, theta):
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
    return _tcheck(tr, lib().gcin_trainer_set_params(tr, _fptr(t), t.size))


def gcin_trainer_forward(tr, ctxs) -> np.ndarray:
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    rows = sum(amg_num_levels(c) for c in ctxs)
    out = np.zeros((rows, 5))
    _tcheck(tr, lib().gcin_trainer_forward(tr, len(ctxs), arr, _dptr(out)))
    return out


def gcin_trainer_backward(tr, dc) -> np.ndarray:
    dc = np.ascontiguousarray(np.asarray(dc, dtype=np.float64))
    g = np.zeros(tr.n_params)
    _tcheck(tr, lib().gcin_trainer_backward(tr, _dptr(dc), _dptr(g)))
    return g


def gcin_trainer_adam_step(tr, lr=1e-3, max_norm=1.0):
    return _tcheck(tr, lib().gcin_trainer_adam_step(tr, float(lr), float(max_norm)))

"""Thin ctypes binding of include/tm.h (argument marshalling only).

Every function has the C name and returns what the C call fills in; a non-zero
tm_status raises TMError carrying the status and tm_last_error().  Pointers may
be given as torch tensors, numpy arrays, ctypes objects or plain integers.
Streams default to torch's current CUDA stream.  There is no fallback: if the
shared library cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtm.so")

TM_OK, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_OOM, TM_ERR_STALE, TM_ERR_NOT_CONVERGED, \
    TM_ERR_BREAKDOWN, TM_ERR_TIMEOUT, TM_ERR_UNSUPPORTED = range(9)
TM_F64, TM_F32, TM_BF16, TM_F16 = range(4)
TM_QHAT_PLUS, TM_QHAT_MINUS, TM_MDAGM, TM_QPQM, TM_QH, TM_QH_DAG, TM_QH_SQ, TM_WHAT_PLUS, TM_WHAT_MINUS, \
    TM_WHAT_SQ = range(10)

PREC_NAMES = {TM_F64: "f64", TM_F32: "f32", TM_BF16: "bf16", TM_F16: "f16"}
STATUS_NAMES = {0: "TM_OK", 1: "TM_ERR_ARG", 2: "TM_ERR_CUDA", 3: "TM_ERR_OOM", 4: "TM_ERR_STALE",
                5: "TM_ERR_NOT_CONVERGED", 6: "TM_ERR_BREAKDOWN", 7: "TM_ERR_TIMEOUT",
                8: "TM_ERR_UNSUPPORTED"}


class tm_params(ct.Structure):
    _fields_ = [("kappa", ct.c_double), ("csw", ct.c_double), ("mu", ct.c_double),
                ("mubar", ct.c_double), ("epsbar", ct.c_double), ("bc_t", ct.c_int), ("rho", ct.c_double)]


class tm_solve_params(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("maxiter", ct.c_int), ("sloppy", ct.c_int),
                ("delta", ct.c_double), ("chunk", ct.c_int), ("use_graph", ct.c_int), ("refine", ct.c_int),
                ("fp64_updates", ct.c_int)]


class tm_solve_info(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("reliable_updates", ct.c_int), ("status", ct.c_int),
                ("true_rel_res", ct.c_double), ("seconds", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tm_tuning(ct.Structure):
    _fields_ = [("even_pass", ct.c_int), ("odd_pass", ct.c_int)]


class tm_mg_params(ct.Structure):
    _fields_ = [("block", ct.c_int * 4), ("nvec", ct.c_int), ("setup_steps", ct.c_int), ("smooth_steps", ct.c_int),
                ("sign", ct.c_int), ("prec", ct.c_int), ("coarse_tol", ct.c_double), ("coarse_maxiter", ct.c_int),
                ("coarse_restart", ct.c_int)]


class TMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2212_06635_gb300.build")
    return ct.CDLL(LIB_PATH)


lib = _load()
_vp = ct.c_void_p
_sigs = {
    "tm_create": [ct.POINTER(_vp), ct.POINTER(ct.c_int), ct.c_int],
    "tm_destroy": [_vp],
    "tm_gauge_load": [_vp, _vp, ct.c_double, _vp],
    "tm_gauge_id": [_vp, ct.POINTER(ct.c_double)],
    "tm_clover_compute": [_vp, ct.POINTER(tm_params), _vp],
    "tm_clover_export": [_vp, ct.c_int, _vp, _vp],
    "tm_field_bytes": [_vp, ct.c_int, ct.c_int, ct.POINTER(ct.c_size_t)],
    "tm_field_import": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_field_export": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_apply_Mhat": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_apply_Mhat_dw": [_vp, ct.c_int, _vp, _vp, _vp],
    "tm_solve_cg": [_vp, ct.c_int, ct.POINTER(tm_solve_params), _vp, _vp, ct.POINTER(tm_solve_info), _vp],
    "tm_solve_multishift": [_vp, ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(_vp), _vp,
                            ct.POINTER(tm_solve_params), ct.POINTER(tm_solve_info), _vp],
    "tm_solve_batch": [ct.POINTER(_vp), ct.c_int, ct.c_int, ct.POINTER(tm_solve_params), ct.POINTER(_vp),
                       ct.POINTER(_vp), ct.POINTER(tm_solve_info), _vp],
    "tm_power_iteration": [_vp, ct.c_int, ct.c_int, ct.POINTER(ct.c_double), _vp],
    "tm_kernel_times": [_vp, ct.c_int, ct.c_int, _vp, ct.c_int, ct.POINTER(ct.c_double), _vp],
    "tm_force_outer": [_vp, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(ct.c_double), ct.POINTER(_vp),
                       ct.POINTER(_vp), ct.c_int, _vp, _vp],
    "tm_apply_even": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_rational_inv_sqrt": [ct.c_int, ct.c_double, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                             ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)],
    "tm_rational_apply": [_vp, ct.c_int, ct.c_int, ct.c_double, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                          _vp, _vp, ct.POINTER(tm_solve_params), ct.POINTER(tm_solve_info), _vp],
    "tm_rational_correction": [_vp, ct.c_int, ct.c_int, ct.c_double, ct.POINTER(ct.c_double),
                               ct.POINTER(ct.c_double), ct.c_double, ct.c_double, _vp, _vp,
                               ct.POINTER(tm_solve_params), ct.POINTER(tm_solve_info), ct.POINTER(ct.c_int), _vp],
    "tm_field_norm2": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_field_norm2_noalloc": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_ptc_create": [ct.POINTER(_vp), ct.c_int, ct.POINTER(ct.c_int), ct.c_int],
    "tm_ptc_destroy": [_vp],
    "tm_ptc_num_weights": [_vp, ct.POINTER(ct.c_size_t)],
    "tm_ptc_set_weights": [_vp, _vp],
    "tm_ptc_init": [_vp, ct.c_double, ct.c_double, ct.c_ulonglong],
    "tm_ptc_get_weights": [_vp, _vp],
    "tm_ptc_apply": [_vp, _vp, _vp, _vp, _vp],
    "tm_ptc_sync": [_vp, _vp],
    "tm_wait_selftest": [ct.c_int, ct.c_double, ct.POINTER(ct.c_int)],
    "tm_ptc_grad": [_vp, _vp, _vp, _vp, ct.POINTER(ct.c_double), _vp, _vp],
    "tm_ptc_train": [_vp, ct.POINTER(_vp), ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_ulonglong,
                     _vp, _vp],
    "tm_ptc_save": [_vp, ct.c_char_p],
    "tm_ptc_load": [_vp, ct.c_char_p],
    "tm_solve_fcg": [_vp, ct.c_int, _vp, ct.POINTER(tm_solve_params), _vp, _vp, ct.POINTER(tm_solve_info), _vp],
    "tm_apply_full": [_vp, ct.c_int, ct.c_int, _vp, _vp, _vp],
    "tm_fma_rate": [ct.c_int, ct.c_int, ct.POINTER(ct.c_double)],
    "tm_mg_create": [ct.POINTER(_vp), _vp, ct.POINTER(tm_mg_params)],
    "tm_mg_destroy": [_vp],
    "tm_mg_coarse_size": [_vp, ct.POINTER(ct.c_size_t)],
    "tm_mg_setup": [_vp, _vp, _vp],
    "tm_mg_vectors": [_vp, _vp, _vp],
    "tm_mg_prolong": [_vp, _vp, _vp, _vp],
    "tm_mg_restrict": [_vp, _vp, _vp, _vp],
    "tm_mg_coarse_apply": [_vp, _vp, _vp, _vp],
    "tm_mg_precondition": [_vp, _vp, _vp, ct.POINTER(ct.c_int), _vp],
    "tm_solve_gcr": [_vp, ct.c_int, _vp, ct.POINTER(tm_solve_params), _vp, _vp, ct.POINTER(tm_solve_info), _vp],
    "tm_autotune": [_vp, ct.c_int, ct.c_int, ct.POINTER(tm_tuning), _vp],
    "tm_set_tuning": [_vp, ct.c_int, ct.c_int, ct.POINTER(tm_tuning)],
    "tm_get_tuning": [_vp, ct.c_int, ct.c_int, ct.POINTER(tm_tuning)],
}
for _n, _a in _sigs.items():
    getattr(lib, _n).argtypes = _a
    getattr(lib, _n).restype = ct.c_int
lib.tm_last_error.argtypes = []
lib.tm_last_error.restype = ct.c_char_p

EXPORTED = list(_sigs) + ["tm_last_error"]


def tm_last_error() -> str:
    return lib.tm_last_error().decode()


def _check(status):
    if status != TM_OK:
        raise TMError(status, tm_last_error())


def ptr(x):
    """Address of a tensor / array / ctypes object / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C contiguous")
        return x.ctypes.data
    return ct.addressof(x)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return stream


def tm_create(dims, device=0):
    h = _vp()
    d = (ct.c_int * 4)(*[int(v) for v in dims])
    _check(lib.tm_create(ct.byref(h), d, int(device)))
    return h.value


def tm_destroy(ctx):
    _check(lib.tm_destroy(ctx))


def tm_gauge_load(ctx, links, gauge_id=0.0, stream=None):
    _check(lib.tm_gauge_load(ctx, ptr(links), float(gauge_id), _stream(stream)))


def tm_gauge_id(ctx):
    v = ct.c_double()
    _check(lib.tm_gauge_id(ctx, ct.byref(v)))
    return v.value


def tm_clover_compute(ctx, kappa, csw, mu=0.0, mubar=0.0, epsbar=0.0, bc_t=-1, rho=0.0, stream=None):
    p = tm_params(kappa, csw, mu, mubar, epsbar, int(bc_t), float(rho))
    _check(lib.tm_clover_compute(ctx, ct.byref(p), _stream(stream)))


def tm_clover_export(ctx, parity, out, stream=None):
    _check(lib.tm_clover_export(ctx, int(parity), ptr(out), _stream(stream)))


def tm_field_bytes(ctx, prec, nflavour=1):
    n = ct.c_size_t()
    _check(lib.tm_field_bytes(ctx, int(prec), int(nflavour), ct.byref(n)))
    return n.value


def tm_field_import(ctx, prec, nflavour, dst, src, stream=None):
    _check(lib.tm_field_import(ctx, int(prec), int(nflavour), ptr(dst), ptr(src), _stream(stream)))


def tm_field_export(ctx, prec, nflavour, dst, src, stream=None):
    _check(lib.tm_field_export(ctx, int(prec), int(nflavour), ptr(dst), ptr(src), _stream(stream)))


def tm_field_norm2(ctx, prec, nflavour, field, result, stream=None):
    """result: device tensor with at least one float64 element."""
    _check(lib.tm_field_norm2(ctx, int(prec), int(nflavour), ptr(field), ptr(result), _stream(stream)))


def tm_field_norm2_noalloc(ctx, prec, nflavour, field, result, stream=None):
    """Allocation-free tm_field_norm2 (see include/tm.h); result: device float64 tensor."""
    _check(lib.tm_field_norm2_noalloc(ctx, int(prec), int(nflavour), ptr(field), ptr(result), _stream(stream)))


def tm_apply_Mhat(ctx, op, prec, out, inp, stream=None):
    _check(lib.tm_apply_Mhat(ctx, int(op), int(prec), ptr(out), ptr(inp), _stream(stream)))


def tm_apply_Mhat_dw(ctx, op, out, inp, stream=None):
    """out = op(inp) on native FP64 fields in double-word arithmetic."""
    _check(lib.tm_apply_Mhat_dw(ctx, int(op), ptr(out), ptr(inp), _stream(stream)))


def tm_apply_even(ctx, op, prec, out, inp, stream=None):
    """out (even sites) = M_ee(s)^-1 H_eo inp (odd sites), s the sign of op."""
    _check(lib.tm_apply_even(ctx, int(op), int(prec), ptr(out), ptr(inp), _stream(stream)))


def solve_params(tol=1e-10, maxiter=100000, sloppy=TM_F64, delta=0.0, chunk=16, use_graph=1, refine=TM_F64,
                 fp64_updates=0):
    """refine: multishift refinement storage precision (TM_F64 = same as sloppy);
    delta <= 0: the library's reliable-update threshold for the sloppy precision;
    fp64_updates: reliable-update residuals with the native FP64 operator."""
    return tm_solve_params(tol, maxiter, sloppy, delta, chunk, use_graph, refine, int(fp64_updates))


def tm_solve_cg(ctx, op, sp, x, b, stream=None, check=True):
    info = tm_solve_info()
    st = lib.tm_solve_cg(ctx, int(op), ct.byref(sp), ptr(x), ptr(b), ct.byref(info), _stream(stream))
    if check:
        _check(st)
    return info


def tm_solve_multishift(ctx, op, shifts, xs, b, sp, stream=None, check=True):
    n = len(shifts)
    sh = (ct.c_double * n)(*shifts)
    xp = (_vp * n)(*[ptr(x) for x in xs])
    infos = (tm_solve_info * n)()
    st = lib.tm_solve_multishift(ctx, int(op), n, sh, xp, ptr(b), ct.byref(sp), infos, _stream(stream))
    if check:
        _check(st)
    return list(infos)


def tm_rational_inv_sqrt(n, lo, hi):
    """(a0, a[n], sigma[n], delta): Zolotarev's r(x) = a0 + sum a_k / (x + sigma_k) ~ x^-1/2 on [lo, hi]."""
    a0 = ct.c_double()
    a = (ct.c_double * n)()
    s = (ct.c_double * n)()
    d = ct.c_double()
    _check(lib.tm_rational_inv_sqrt(int(n), float(lo), float(hi), ct.byref(a0), a, s, ct.byref(d)))
    return a0.value, list(a), list(s), d.value


def tm_rational_apply(ctx, op, coeffs, y, b, sp, stream=None, check=True):
    """y = r(A) b for coeffs = (a0, a, sigma[, ...])."""
    a0, a, sigma = coeffs[0], coeffs[1], coeffs[2]
    n = len(a)
    ap = (ct.c_double * n)(*a)
    sg = (ct.c_double * n)(*sigma)
    infos = (tm_solve_info * n)()
    st = lib.tm_rational_apply(ctx, int(op), n, float(a0), ap, sg, ptr(y), ptr(b), ct.byref(sp), infos,
                               _stream(stream))
    if check:
        _check(st)
    return list(infos)


def tm_rational_correction(ctx, op, coeffs, p, y, b, sp, series_tol=1e-14, stream=None, check=True):
    """y = (1 + Z)^p b, Z = A r(A)^2 - 1; returns (infos, number of Z applications)."""
    a0, a, sigma = coeffs[0], coeffs[1], coeffs[2]
    n = len(a)
    ap = (ct.c_double * n)(*a)
    sg = (ct.c_double * n)(*sigma)
    infos = (tm_solve_info * n)()
    na = ct.c_int()
    st = lib.tm_rational_correction(ctx, int(op), n, float(a0), ap, sg, float(p), float(series_tol), ptr(y),
                                    ptr(b), ct.byref(sp), infos, ct.byref(na), _stream(stream))
    if check:
        _check(st)
    return list(infos), na.value


def tm_solve_batch(ctxs, op, sp, xs, bs, stream=None, check=True):
    n = len(ctxs)
    cp = (_vp * n)(*ctxs)
    xp = (_vp * n)(*[ptr(x) for x in xs])
    bp = (_vp * n)(*[ptr(b) for b in bs])
    infos = (tm_solve_info * n)()
    st = lib.tm_solve_batch(cp, n, int(op), ct.byref(sp), xp, bp, infos, _stream(stream))
    if check:
        _check(st)
    return list(infos)


def tm_power_iteration(ctx, op, iters=100, stream=None):
    v = ct.c_double()
    _check(lib.tm_power_iteration(ctx, int(op), int(iters), ct.byref(v), _stream(stream)))
    return v.value


def tm_kernel_times(ctx, op, prec, inp, reps=20, stream=None):
    ms = (ct.c_double * 2)()
    _check(lib.tm_kernel_times(ctx, int(op), int(prec), ptr(inp), int(reps), ms, _stream(stream)))
    return ms[0], ms[1]


TM_FORCE_MAXN = 32


def tm_force_outer(ctx, prec, nflavour, coeffs, xs, ys, force, gamma5_y=False, stream=None, check=True):
    """force += T_A[U W] on every link for the field pairs (X_k, Y_k) with weights
    coeffs[k]; xs[k], ys[k] = (even-parity native field, odd-parity native field);
    gamma5_y: the Y fields enter as g5 Y_k."""
    n = len(coeffs)
    if len(xs) != n or len(ys) != n:
        raise ValueError("one (even, odd) field pair of X and of Y per weight")
    cf = (ct.c_double * max(n, 1))(*coeffs)
    xp = (_vp * max(2 * n, 1))(*[ptr(f) for pair in xs for f in pair])
    yp = (_vp * max(2 * n, 1))(*[ptr(f) for pair in ys for f in pair])
    st = lib.tm_force_outer(ctx, int(prec), int(nflavour), n, cf, xp, yp, int(bool(gamma5_y)), ptr(force),
                            _stream(stream))
    if check:
        _check(st)
    return st


def tm_autotune(ctx, prec, nflavour=1, stream=None):
    t = tm_tuning()
    _check(lib.tm_autotune(ctx, int(prec), int(nflavour), ct.byref(t), _stream(stream)))
    return t.even_pass, t.odd_pass


def tm_set_tuning(ctx, prec, nflavour, even_pass, odd_pass):
    t = tm_tuning(int(even_pass), int(odd_pass))
    _check(lib.tm_set_tuning(ctx, int(prec), int(nflavour), ct.byref(t)))


def tm_get_tuning(ctx, prec, nflavour=1):
    t = tm_tuning()
    _check(lib.tm_get_tuning(ctx, int(prec), int(nflavour), ct.byref(t)))
    return t.even_pass, t.odd_pass


# --- learned preconditioner ----------------------------------------------------
def tm_ptc_create(channels, device=0):
    h = _vp()
    ch = (ct.c_int * len(channels))(*[int(c) for c in channels])
    _check(lib.tm_ptc_create(ct.byref(h), len(channels) - 1, ch, int(device)))
    return h.value


def tm_ptc_destroy(net):
    _check(lib.tm_ptc_destroy(net))


def tm_ptc_num_weights(net):
    n = ct.c_size_t()
    _check(lib.tm_ptc_num_weights(net, ct.byref(n)))
    return n.value


def tm_ptc_set_weights(net, w):
    """w: complex128 array, canonical layout, flattened in layer order."""
    a = np.ascontiguousarray(w, dtype=np.complex128)
    _check(lib.tm_ptc_set_weights(net, a.ctypes.data))


def tm_ptc_init(net, scale=0.5, noise=0.01, seed=4000):
    _check(lib.tm_ptc_init(net, float(scale), float(noise), int(seed)))


def tm_ptc_get_weights(net):
    a = np.empty(tm_ptc_num_weights(net), dtype=np.complex128)
    _check(lib.tm_ptc_get_weights(net, a.ctypes.data))
    return a


def tm_ptc_apply(net, ctx, out, inp, stream=None):
    _check(lib.tm_ptc_apply(net, ctx, ptr(out), ptr(inp), _stream(stream)))


def tm_wait_selftest(seconds=1e-3, device=0):
    """Bounded-wait check: returns 1 when a wait on an mbarrier nobody arrives on ran out."""
    out = ct.c_int(-1)
    _check(lib.tm_wait_selftest(device, seconds, ct.byref(out)))
    return out.value


def tm_ptc_sync(net, stream=None):
    _check(lib.tm_ptc_sync(net, _stream(stream)))


def tm_ptc_grad(net, ctx, r, e, stream=None):
    loss = ct.c_double()
    g = np.empty(tm_ptc_num_weights(net), dtype=np.complex128)
    _check(lib.tm_ptc_grad(net, ctx, ptr(r), ptr(e), ct.byref(loss), g.ctypes.data, _stream(stream)))
    return loss.value, g


def tm_ptc_train(net, ctxs, op, npairs, batch=1, lr=1e-3, seed=5000, stream=None):
    cp = (_vp * len(ctxs))(*ctxs)
    losses = np.empty(npairs, dtype=np.float64)
    _check(lib.tm_ptc_train(net, cp, len(ctxs), int(op), int(npairs), int(batch), float(lr), int(seed),
                            losses.ctypes.data, _stream(stream)))
    return losses


def tm_ptc_save(net, path):
    _check(lib.tm_ptc_save(net, str(path).encode()))


def tm_ptc_load(net, path):
    _check(lib.tm_ptc_load(net, str(path).encode()))


def tm_solve_fcg(ctx, op, net, sp, x, b, stream=None, check=True):
    info = tm_solve_info()
    st = lib.tm_solve_fcg(ctx, int(op), net, ct.byref(sp), ptr(x), ptr(b), ct.byref(info), _stream(stream))
    if check:
        _check(st)
    return info


# ---------------------------------------------------------------------------
# two-level multigrid on the full operator
# ---------------------------------------------------------------------------
def mg_params(block, nvec, setup_steps=20, smooth_steps=4, sign=1, prec=TM_F32, coarse_tol=0.05,
              coarse_maxiter=200, coarse_restart=16):
    return tm_mg_params((ct.c_int * 4)(*block), nvec, setup_steps, smooth_steps, sign, prec, coarse_tol,
                        coarse_maxiter, coarse_restart)


def tm_apply_full(ctx, sign, prec, out, inp, stream=None):
    _check(lib.tm_apply_full(ctx, int(sign), int(prec), ptr(out), ptr(inp), _stream(stream)))


def tm_mg_create(ctx, params):
    h = _vp()
    _check(lib.tm_mg_create(ct.byref(h), ctx, ct.byref(params)))
    return h.value


def tm_mg_destroy(mg):
    _check(lib.tm_mg_destroy(mg))


def tm_mg_coarse_size(mg):
    n = ct.c_size_t()
    _check(lib.tm_mg_coarse_size(mg, ct.byref(n)))
    return n.value


def tm_mg_setup(mg, init, stream=None):
    _check(lib.tm_mg_setup(mg, ptr(init), _stream(stream)))


def tm_mg_vectors(mg, out, stream=None):
    _check(lib.tm_mg_vectors(mg, ptr(out), _stream(stream)))


def tm_mg_prolong(mg, fine, coarse, stream=None):
    _check(lib.tm_mg_prolong(mg, ptr(fine), ptr(coarse), _stream(stream)))


def tm_mg_restrict(mg, coarse, fine, stream=None):
    _check(lib.tm_mg_restrict(mg, ptr(coarse), ptr(fine), _stream(stream)))


def tm_mg_coarse_apply(mg, out, inp, stream=None):
    _check(lib.tm_mg_coarse_apply(mg, ptr(out), ptr(inp), _stream(stream)))


def tm_mg_precondition(mg, z, r, stream=None):
    it = ct.c_int()
    _check(lib.tm_mg_precondition(mg, ptr(z), ptr(r), ct.byref(it), _stream(stream)))
    return it.value


def tm_solve_gcr(ctx, sign, mg, sp, x, b, stream=None, check=True):
    info = tm_solve_info()
    st = lib.tm_solve_gcr(ctx, int(sign), mg, ct.byref(sp), ptr(x), ptr(b), ct.byref(info), _stream(stream))
    if check:
        _check(st)
    return info


def tm_fma_rate(device, prec):
    """Measured FMA rate of the CUDA cores, flops per second (FP64 or FP32)."""
    v = ct.c_double()
    _check(lib.tm_fma_rate(int(device), int(prec), ct.byref(v)))
    return v.value

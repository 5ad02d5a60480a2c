"""Python binding of libovl.so, the GB300 overlap-operator library.

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI declared in include/ovl.h. There is no CPU fallback;
if the shared library has not been built, every call raises.

Vectors are complex128 arrays [V][4][3] (or [n_rhs][V][4][3]) in lexicographic
site order, as numpy arrays (host) or torch tensors (host or CUDA); gauge
fields are complex128 [V][4][3][3].
"""

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libovl.so")

OVL_OK, OVL_EINVAL, OVL_ENOMEM, OVL_ENOCONV, OVL_EBREAKDOWN, OVL_ETIMEOUT, OVL_ECUDA = range(7)
OVL_FP64, OVL_MIXED_FP32, OVL_MIXED_HALF, OVL_MIXED_BF16 = range(4)
OVL_PREC_NONE, OVL_PREC_WILSON, OVL_PREC_RECURSIVE = range(3)
OVL_SIGN_ZOLOTAREV, OVL_SIGN_KRYLOV = range(2)
OVL_ARITH_FP64, OVL_ARITH_FF, OVL_ARITH_FP32, OVL_ARITH_FP16, OVL_ARITH_BF16 = range(5)
_STATUS = {0: "OVL_OK", 1: "OVL_EINVAL", 2: "OVL_ENOMEM", 3: "OVL_ENOCONV", 4: "OVL_EBREAKDOWN",
           5: "OVL_ETIMEOUT", 6: "OVL_ECUDA"}


class OvlError(RuntimeError):
    """A non-OK ovl_status, with the library's one-line reason."""

    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class ovl_params(ctypes.Structure):
    """Mirror of ovl_params in include/ovl.h (same fields, same order)."""
    _fields_ = [
        ("tol_outer", ctypes.c_double), ("restart", ctypes.c_int), ("relax", ctypes.c_int),
        ("relax_factor", ctypes.c_double), ("n_poles", ctypes.c_int), ("lambda_min", ctypes.c_double),
        ("lambda_max", ctypes.c_double), ("sign_tol", ctypes.c_double), ("precond", ctypes.c_int),
        ("m0_prec", ctypes.c_double), ("eps_prec", ctypes.c_double), ("eps_inner", ctypes.c_double),
        ("restart_inner", ctypes.c_int), ("max_inner", ctypes.c_int), ("precision", ctypes.c_int),
        ("antiperiodic", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_ms_iter", ctypes.c_int),
        ("sap_block", ctypes.c_int * 4), ("sap_cycles", ctypes.c_int), ("sap_mr_iters", ctypes.c_int),
        ("prec_restart", ctypes.c_int), ("prec_max_iter", ctypes.c_int), ("rhs_block", ctypes.c_int),
        ("use_graphs", ctypes.c_int), ("check_every", ctypes.c_int), ("stencil_tps", ctypes.c_int),
        ("sap_tps", ctypes.c_int), ("adaptive_poles", ctypes.c_int), ("n_deflate", ctypes.c_int),
        ("deflate_tol", ctypes.c_double), ("sign_method", ctypes.c_int), ("krylov_m", ctypes.c_int),
        ("krylov_keep", ctypes.c_int), ("ff_outer", ctypes.c_int), ("max_seconds", ctypes.c_double),
        ("wilson_mg", ctypes.c_int), ("mg_nv", ctypes.c_int), ("mg_setup_iters", ctypes.c_int),
        ("mg_coarse_steps", ctypes.c_int), ("mg_coarse_tol", ctypes.c_double), ("m0_adapt", ctypes.c_int),
        ("mrhs_kernel", ctypes.c_int),
    ]


class ovl_stats(ctypes.Structure):
    """Mirror of ovl_stats (per-solve statistics)."""
    _fields_ = [
        ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int), ("ms_iters_fp64", ctypes.c_long),
        ("ms_iters_low", ctypes.c_long), ("prec_iters", ctypes.c_long), ("true_rel_resid", ctypes.c_double),
        ("seconds", ctypes.c_double), ("t_sign_fp64", ctypes.c_double), ("t_sign_low", ctypes.c_double),
        ("t_prec", ctypes.c_double), ("ms_iters_ff", ctypes.c_long),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ovl_request(ctypes.Structure):
    """Mirror of ovl_request (one serving request)."""
    _fields_ = [("gauge", ctypes.c_void_p), ("gauge_key", ctypes.c_long), ("dims", ctypes.c_int * 4),
                ("rho", ctypes.c_double), ("mu", ctypes.c_double), ("n_rhs", ctypes.c_int),
                ("b", ctypes.c_void_p), ("x", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("params", ctypes.c_void_p)]


class ovl_result(ctypes.Structure):
    """Mirror of ovl_result (a served request's outcome)."""
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("stats", ovl_stats),
                ("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("message", ctypes.c_char * 160)]

    def as_dict(self):
        return {"done": self.done, "status": self.status, "stats": self.stats.as_dict(), "queue_s": self.queue_s,
                "run_s": self.run_s, "latency_s": self.latency_s, "device_bytes": self.device_bytes,
                "message": self.message.decode(errors="replace")}


class ovl_prof_kernel(ctypes.Structure):
    """Mirror of ovl_prof_kernel (counters of one kernel class)."""
    _fields_ = [("ms", ctypes.c_double), ("launches", ctypes.c_long), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double), ("timed", ctypes.c_long), ("timed_bytes", ctypes.c_double)]


PROF_KERNELS = ["ms_stencil_f64", "ms_shifts_f64", "ms_stencil_f32", "ms_shifts_f32", "ms_stencil_ff",
                "ms_shifts_ff"]


class ovl_prof(ctypes.Structure):
    """Mirror of ovl_prof (instrumentation counters)."""
    _fields_ = [("launches", ctypes.c_long), ("k", ovl_prof_kernel * 6), ("valid", ctypes.c_int)]

    def as_dict(self):
        d = {"launches": self.launches, "valid": self.valid}
        for name, k in zip(PROF_KERNELS, self.k):
            d[name] = {"ms": k.ms, "launches": k.launches, "bytes": k.bytes, "flops": k.flops,
                       "timed": k.timed, "timed_bytes": k.timed_bytes}
        return d


EXPORTS = ["ovl_params_default", "ovl_create", "wilson_apply", "sign_apply", "ovl_apply", "ovl_solve",
           "ovl_info", "ovl_zolotarev", "ovl_destroy", "ovl_last_error", "ovl_prof_enable", "ovl_prof_get",
           "wilson_solve", "ovl_tuning", "ovl_tuning_sap", "ovl_hermitian_eig", "ovl_deflation_info", "ovl_krylov_sign_info", "ovl_request_bytes", "wilson_sap_apply", "wilson_apply_noalloc", "ovl_dslash_time", "wilson_apply_n",
           "ovl_apply_n", "ovl_dslash_time_n", "wilson_apply_arith", "wilson_apply_n_arith", "sign_apply_arith", "ovl_fma_peak", "ovl_mg_setup", "wilson_mg_apply", "ovl_mg_info", "ovl_m0_adapt_info", "ovl_tuning_mrhs", "ovl_server_create", "ovl_server_submit", "ovl_server_query",
           "ovl_server_wait", "ovl_server_report", "ovl_server_destroy"]

_lib = None


def lib():
    """Loads libovl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libovl.so not built (%s); run paper_1410_7170_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I_, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.ovl_params_default.argtypes = [ctypes.POINTER(ovl_params)]
        L.ovl_create.argtypes = [ctypes.POINTER(P), P, P, D, D, ctypes.POINTER(ovl_params), P]
        L.wilson_apply.argtypes = [P, P, P, D]
        L.sign_apply.argtypes = [P, P, P, D]
        L.ovl_apply.argtypes = [P, P, P, D]
        L.ovl_solve.argtypes = [P, P, P, I_, D, ctypes.POINTER(ovl_stats)]
        L.ovl_info.argtypes = [P] + [ctypes.POINTER(D)] * 7
        L.ovl_zolotarev.argtypes = [D, I_, ctypes.POINTER(D), P, P, ctypes.POINTER(D)]
        L.ovl_destroy.argtypes = [P]
        L.ovl_last_error.argtypes = [P]
        L.ovl_last_error.restype = ctypes.c_char_p
        L.ovl_prof_enable.argtypes = [P, I_]
        L.ovl_prof_get.argtypes = [P, ctypes.POINTER(ovl_prof), I_]
        L.wilson_solve.argtypes = [P, P, P, D, D, ctypes.POINTER(I_)]
        L.wilson_sap_apply.argtypes = [P, P, P, D]
        L.ovl_tuning.argtypes = [P, ctypes.POINTER(I_), ctypes.POINTER(I_), P]
        L.ovl_tuning_sap.argtypes = [P, ctypes.POINTER(I_), P]
        L.ovl_tuning_mrhs.argtypes = [P, P, P]
        L.ovl_hermitian_eig.argtypes = [I_, P, P, P]
        L.ovl_deflation_info.argtypes = [P, ctypes.POINTER(I_), P, ctypes.POINTER(D), ctypes.POINTER(D),
                                         ctypes.POINTER(D), ctypes.POINTER(ctypes.c_long)]
        L.ovl_request_bytes.argtypes = [ctypes.POINTER(ovl_request), ctypes.POINTER(ctypes.c_size_t)]
        L.ovl_krylov_sign_info.argtypes = [P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]
        L.wilson_apply_noalloc.argtypes = [P, P, P, P, D, I_, P]
        L.ovl_dslash_time.argtypes = [P, I_, I_, ctypes.POINTER(D)]
        L.wilson_apply_n.argtypes = [P, P, P, I_, D]
        L.ovl_apply_n.argtypes = [P, P, P, I_, D]
        L.ovl_dslash_time_n.argtypes = [P, I_, I_, I_, ctypes.POINTER(D)]
        L.wilson_apply_arith.argtypes = [P, P, P, D, I_]
        L.wilson_apply_n_arith.argtypes = [P, P, P, I_, D, I_]
        L.sign_apply_arith.argtypes = [P, P, P, D, I_]
        L.ovl_fma_peak.argtypes = [I_, ctypes.POINTER(D)]
        L.ovl_mg_setup.argtypes = [P, D, P, I_]
        L.wilson_mg_apply.argtypes = [P, P, P, D]
        L.ovl_mg_info.argtypes = [P, ctypes.POINTER(I_), ctypes.POINTER(I_), ctypes.POINTER(I_), ctypes.POINTER(D)]
        L.ovl_m0_adapt_info.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(D)]
        L.ovl_server_create.argtypes = [ctypes.POINTER(P), I_, ctypes.c_size_t]
        L.ovl_server_submit.argtypes = [P, ctypes.POINTER(ovl_request), ctypes.POINTER(ctypes.c_long)]
        L.ovl_server_query.argtypes = [P, ctypes.c_long, ctypes.POINTER(ovl_result)]
        L.ovl_server_wait.argtypes = [P, ctypes.c_long, ctypes.POINTER(ovl_result)]
        L.ovl_server_report.argtypes = [P] + [ctypes.POINTER(D)] * 3 + [ctypes.POINTER(ctypes.c_size_t),
                                                                         ctypes.POINTER(ctypes.c_long),
                                                                         ctypes.POINTER(ctypes.c_long)]
        L.ovl_server_destroy.argtypes = [P]
        for name in EXPORTS:
            if name not in ("ovl_last_error",):
                getattr(L, name).restype = I_
        _lib = L
    return _lib


def _ptr(a, writable=False):
    """Data pointer of a contiguous numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "__array_interface__"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("array must be writable")
        return ctypes.c_void_p(a.__array_interface__["data"][0])
    raise TypeError("expected a numpy array or torch tensor")


def _check(st, ctx=None):
    if st != OVL_OK:
        raise OvlError(st, lib().ovl_last_error(ctx).decode())


def params_default(**kw):
    """ovl_params with the library's defaults (Table 2 / Table 3 values where the paper gives
    one), then the given fields set by name (sap_block as a 4-sequence)."""
    p = ovl_params()
    _check(lib().ovl_params_default(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "sap_block":
            for m in range(4):
                p.sap_block[m] = int(v[m])
        else:
            setattr(p, k, v)
    return p


def ovl_zolotarev(k, n):
    """(d0, a[n], c[n], delta) of the library's host Zolotarev computation."""
    import numpy as np
    a = np.zeros(n)
    c = np.zeros(n)
    d0 = ctypes.c_double()
    delta = ctypes.c_double()
    _check(lib().ovl_zolotarev(float(k), int(n), ctypes.byref(d0), _ptr(a), _ptr(c), ctypes.byref(delta)))
    return d0.value, a, c, delta.value


def ovl_create(gauge, dims, rho, mu, params=None, stream=None):
    """New context for D_N with kernel mass -rho and overlap mass mu on the lattice dims;
    gauge: [V][4][3][3] complex128 (host or device); stream: a cudaStream_t handle or None."""
    ctx = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    st = lib().ovl_create(ctypes.byref(ctx), _ptr(gauge), ctypes.cast(d, ctypes.c_void_p), float(rho),
                          float(mu), ctypes.byref(params) if params is not None else None,
                          ctypes.c_void_p(stream) if stream else None)
    _check(st, None)
    return ctx


def ovl_destroy(ctx):
    """Frees the context and its device memory (None is a no-op)."""
    if ctx:
        _check(lib().ovl_destroy(ctx))


def wilson_apply(ctx, out, inp, m0):
    """out = D_W(m0) inp (Eq. Wilson-Dirac); [V][4][3] complex128 buffers, host or device."""
    _check(lib().wilson_apply(ctx, _ptr(out, True), _ptr(inp), float(m0)), ctx)
    return out


def sign_apply(ctx, out, inp, tol):
    """out ~= sign(Gamma5 D_W(m0_ker)) inp to relative accuracy tol (FP64)."""
    _check(lib().sign_apply(ctx, _ptr(out, True), _ptr(inp), float(tol)), ctx)
    return out


def wilson_apply_arith(ctx, out, inp, m0, arith):
    """out = D_W(m0) inp in the arithmetic `arith` (OVL_ARITH_FP64, OVL_ARITH_FF or OVL_ARITH_FP32)."""
    _check(lib().wilson_apply_arith(ctx, _ptr(out, True), _ptr(inp), float(m0), int(arith)), ctx)
    return out


def wilson_apply_n_arith(ctx, out, inp, n_rhs, m0, arith):
    """out_k = D_W(m0) inp_k with the multi-RHS stencil in OVL_ARITH_FP64 or OVL_ARITH_FP32."""
    _check(lib().wilson_apply_n_arith(ctx, _ptr(out, True), _ptr(inp), int(n_rhs), float(m0), int(arith)), ctx)
    return out


def sign_apply_arith(ctx, out, inp, tol, arith):
    """out ~= sign(Q) inp to accuracy tol in any ovl_arith (FP64, FF, FP32, FP16- or BF16-stored)."""
    _check(lib().sign_apply_arith(ctx, _ptr(out, True), _ptr(inp), float(tol), int(arith)), ctx)
    return out


def ovl_mg_setup(ctx, m0, start=None, n_start=0):
    """Builds the two-level multigrid for D_W(m0); start: [n][V][4][3] start vectors or None."""
    _check(lib().ovl_mg_setup(ctx, float(m0), _ptr(start) if start is not None else None,
                              int(n_start if start is not None else 0)), ctx)


def wilson_mg_apply(ctx, out, inp, m0):
    """out = M_MG inp: one application of the two-level multigrid preconditioner for D_W(m0)."""
    _check(lib().wilson_mg_apply(ctx, _ptr(out, True), _ptr(inp), float(m0)), ctx)
    return out


def ovl_mg_info(ctx):
    """Test vectors, coarse sites, GMRES steps of the last coarse solve, setup seconds."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    d = ctypes.c_double()
    _check(lib().ovl_mg_info(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), ctx)
    return {"nv": a.value, "coarse_sites": b.value, "last_coarse_steps": c.value, "setup_s": d.value}


def ovl_m0_adapt_info(ctx):
    """Candidate preconditioner masses, their scores, applications so far and the best mass."""
    import numpy as np
    cand = np.zeros(5)
    eff = np.zeros(5)
    uses, best = ctypes.c_long(), ctypes.c_double()
    _check(lib().ovl_m0_adapt_info(ctx, _ptr(cand, True), _ptr(eff, True), ctypes.byref(uses), ctypes.byref(best)), ctx)
    return {"cand": cand.tolist(), "eff": eff.tolist(), "uses": uses.value, "best": best.value}


def ovl_apply(ctx, out, inp, tol):
    """out ~= D_N inp = rho inp + Gamma5 sign(Q) inp (Eq. overlap_def), sign to accuracy tol."""
    _check(lib().ovl_apply(ctx, _ptr(out, True), _ptr(inp), float(tol)), ctx)
    return out


def ovl_solve(ctx, x, b, n_rhs=1, tol=0.0, check=True):
    """Solves D_N x = b in place on x; returns (status, stats dict)."""
    s = ovl_stats()
    st = lib().ovl_solve(ctx, _ptr(x, True), _ptr(b), int(n_rhs), float(tol), ctypes.byref(s))
    if check and st != OVL_OK:
        _check(st, ctx)
    return st, s.as_dict()


def wilson_apply_noalloc(out, inp, gauge, dims, m0, antiperiodic=True, stream=None):
    """out = D_W(m0) inp without a context and without device allocation (device tensors only).

    The C entry point cannot see buffer sizes, so the sizes, dtype, layout and device of the
    three tensors are checked here before the call. Returns once the work is enqueued on
    `stream` (default: the legacy default stream)."""
    V = int(math.prod(int(x) for x in dims))
    for name, t, n in (("out", out, V * 12), ("inp", inp, V * 12), ("gauge", gauge, V * 36)):
        if hasattr(t, "data_ptr"):
            import torch
            if t.dtype != torch.complex128 or not t.is_contiguous():
                raise ValueError("%s must be a contiguous complex128 tensor" % name)
            if t.numel() < n:
                raise ValueError("%s holds %d complex numbers, needs %d" % (name, t.numel(), n))
            if t.is_cuda and t.device.index != torch.cuda.current_device():
                raise ValueError("%s is on cuda:%d, the current device is cuda:%d"
                                 % (name, t.device.index, torch.cuda.current_device()))
        elif getattr(t, "size", n) < n:
            raise ValueError("%s holds %d complex numbers, needs %d" % (name, t.size, n))
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    _check(lib().wilson_apply_noalloc(_ptr(out, True), _ptr(inp), _ptr(gauge), ctypes.cast(d, ctypes.c_void_p),
                                      float(m0), int(bool(antiperiodic)),
                                      ctypes.c_void_p(stream) if stream else None), None)
    return out


def wilson_sap_apply(ctx, out, inp, m0):
    """out = M_SAP inp: one application of the Schwarz preconditioner on D_W(m0)."""
    _check(lib().wilson_sap_apply(ctx, _ptr(out, True), _ptr(inp), float(m0)), ctx)
    return out


def wilson_solve(ctx, x, b, m0, tol):
    """x ~ D_W(m0)^{-1} b (SAP-preconditioned FGMRES); returns the iteration count."""
    it = ctypes.c_int()
    _check(lib().wilson_solve(ctx, _ptr(x, True), _ptr(b), float(m0), float(tol), ctypes.byref(it)), ctx)
    return it.value


def ovl_tuning(ctx):
    """Stencil threads per site chosen by the autotuner (FP64, FP32) and the timed variants (ms)."""
    import numpy as np
    a, b = ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(4, dtype=np.float32)
    _check(lib().ovl_tuning(ctx, ctypes.byref(a), ctypes.byref(b), _ptr(ms)), ctx)
    return {"tps64": a.value, "tps32": b.value, "ms": ms.tolist()}


def hermitian_eig(A):
    """Eigenvalues (ascending) and eigenvectors (columns) of a complex Hermitian matrix (host)."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.empty(n)
    Z = np.empty((n, n), dtype=np.complex128)
    _check(lib().ovl_hermitian_eig(int(n), _ptr(A), _ptr(w, True), _ptr(Z, True)))
    return w, Z


def ovl_deflation_info(ctx):
    """Deflated eigenvalues of Q, |lambda_{k+1}|, setup seconds, worst eigenpair residual and the
    eigensolver's Q^2 products (k = 0 without deflation)."""
    import numpy as np
    k = ctypes.c_int()
    _check(lib().ovl_deflation_info(ctx, ctypes.byref(k), None, None, None, None, None), ctx)
    lam = np.zeros(max(k.value, 1))
    nxt, t, res, mv = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_long()
    _check(lib().ovl_deflation_info(ctx, None, _ptr(lam, True), ctypes.byref(nxt), ctypes.byref(t),
                                    ctypes.byref(res), ctypes.byref(mv)), ctx)
    return {"k": k.value, "lambda": lam[:k.value].tolist(), "lambda_next": nxt.value, "setup_s": t.value,
            "resid_max": res.value, "matvecs": mv.value}


def request_bytes(dims, n_rhs=1, params=None):
    """Device bytes the serving loop reserves for a request (host-side estimate, no GPU)."""
    req = ovl_request()
    for m in range(4):
        req.dims[m] = int(dims[m])
    req.n_rhs = int(n_rhs)
    req.params = ctypes.cast(ctypes.byref(params), ctypes.c_void_p).value if params is not None else None
    out = ctypes.c_size_t()
    _check(lib().ovl_request_bytes(ctypes.byref(req), ctypes.byref(out)))
    return out.value


def ovl_krylov_sign_info(ctx):
    """Cycles and Q^2 products of the restarted Krylov sign function since the context was made."""
    cyc, mv = ctypes.c_long(), ctypes.c_long()
    _check(lib().ovl_krylov_sign_info(ctx, ctypes.byref(cyc), ctypes.byref(mv)), ctx)
    return {"cycles": cyc.value, "matvecs": mv.value}


def ovl_tuning_mrhs(ctx):
    """FP32 multi-RHS stencil kernels chosen for this lattice shape (1 RHS pairs, 2 tiles of 32
    sites, 3 staged links) for blocks of up to 6 and of 7..12 right-hand sides, and the timed ms
    per right-hand side of each candidate at 4 and at 12."""
    import numpy as np
    k = np.zeros(2, dtype=np.int32)
    ms = np.zeros(6, dtype=np.float32)
    _check(lib().ovl_tuning_mrhs(ctx, _ptr(k), _ptr(ms)), ctx)
    return {"kernel": int(k[0]), "kernel_large": int(k[1]), "ms4": ms[:3].tolist(), "ms12": ms[3:].tolist()}


def ovl_tuning_sap(ctx):
    """Threads per block site of the FP32 Schwarz block solves and the timed variants (ms)."""
    import numpy as np
    a = ctypes.c_int()
    ms = np.zeros(3, dtype=np.float32)
    _check(lib().ovl_tuning_sap(ctx, ctypes.byref(a), _ptr(ms)), ctx)
    return {"sap_tps": a.value, "ms": ms.tolist()}


def ovl_dslash_time(ctx, precision, reps=20):
    """Average ms of one full-lattice Wilson stencil launch (precision 0 = FP64, 1 = FP32,
    2 = float-float) on a seeded random input."""
    ms = ctypes.c_double()
    _check(lib().ovl_dslash_time(ctx, int(precision), int(reps), ctypes.byref(ms)), ctx)
    return ms.value


def wilson_apply_n(ctx, out, inp, n_rhs, m0):
    """out_k = D_W(m0) inp_k for n_rhs vectors back to back (multi-RHS stencil)."""
    _check(lib().wilson_apply_n(ctx, _ptr(out, True), _ptr(inp), int(n_rhs), float(m0)), ctx)
    return out


def ovl_apply_n(ctx, out, inp, n_rhs, tol):
    """out_k ~= D_N inp_k for n_rhs vectors back to back (lock-step batched multishift)."""
    _check(lib().ovl_apply_n(ctx, _ptr(out, True), _ptr(inp), int(n_rhs), float(tol)), ctx)
    return out


def ovl_dslash_time_n(ctx, precision, nrhs, reps=20):
    """ms per launch of the multi-RHS stencil on nrhs right-hand sides (0 = FP64, 1 = FP32)."""
    ms = ctypes.c_double()
    _check(lib().ovl_dslash_time_n(ctx, int(precision), int(nrhs), int(reps), ctypes.byref(ms)), ctx)
    return ms.value


def fma_peak(precision):
    """Measured FMA throughput of the current GPU in GFLOP/s (precision 0 = FP64, 1 = FP32)."""
    g = ctypes.c_double()
    _check(lib().ovl_fma_peak(int(precision), ctypes.byref(g)))
    return g.value


def ovl_info(ctx):
    """Spectral interval of |Q|, Zolotarev error bound, rho, m0_ker, m0_prec and sigma_min."""
    vals = [ctypes.c_double() for _ in range(7)]
    _check(lib().ovl_info(ctx, *[ctypes.byref(v) for v in vals]), ctx)
    keys = ["lambda_min", "lambda_max", "delta", "rho", "m0_ker", "m0_prec", "sigma_min"]
    return {k: v.value for k, v in zip(keys, vals)}


def ovl_prof_enable(ctx, on=True):
    """Switches the multishift event instrumentation on or off."""
    _check(lib().ovl_prof_enable(ctx, int(bool(on))), ctx)


def ovl_prof_get(ctx, reset=False):
    """Instrumentation counters per kernel class (launches, timed ms, algorithmic bytes/flops)."""
    out = ovl_prof()
    _check(lib().ovl_prof_get(ctx, ctypes.byref(out), int(bool(reset))), ctx)
    return out.as_dict()


class Overlap:
    """Owns one library context (ovl_create ... ovl_destroy)."""

    def __init__(self, gauge, dims, rho, mu, params=None, stream=None):
        self.dims = tuple(int(x) for x in dims)
        self.V = int(math.prod(self.dims))
        self.ctx = ovl_create(gauge, self.dims, rho, mu, params, stream)

    def close(self):
        if self.ctx:
            ovl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def wilson_apply(self, out, inp, m0):
        return wilson_apply(self.ctx, out, inp, m0)

    def sign_apply(self, out, inp, tol):
        return sign_apply(self.ctx, out, inp, tol)

    def ovl_apply(self, out, inp, tol):
        return ovl_apply(self.ctx, out, inp, tol)

    def mg_setup(self, m0, start=None):
        return ovl_mg_setup(self.ctx, m0, start, 0 if start is None else len(start))

    def mg_apply(self, out, inp, m0):
        return wilson_mg_apply(self.ctx, out, inp, m0)

    def mg_info(self):
        return ovl_mg_info(self.ctx)

    def m0_adapt_info(self):
        return ovl_m0_adapt_info(self.ctx)

    def wilson_apply_arith(self, out, inp, m0, arith):
        return wilson_apply_arith(self.ctx, out, inp, m0, arith)

    def wilson_apply_n_arith(self, out, inp, n_rhs, m0, arith):
        return wilson_apply_n_arith(self.ctx, out, inp, n_rhs, m0, arith)

    def sign_apply_arith(self, out, inp, tol, arith):
        return sign_apply_arith(self.ctx, out, inp, tol, arith)

    def ovl_solve(self, x, b, n_rhs=1, tol=0.0, check=True):
        return ovl_solve(self.ctx, x, b, n_rhs, tol, check)

    def info(self):
        return ovl_info(self.ctx)

    def wilson_solve(self, x, b, m0, tol):
        return wilson_solve(self.ctx, x, b, m0, tol)

    def sap_apply(self, out, inp, m0):
        return wilson_sap_apply(self.ctx, out, inp, m0)

    def tuning(self):
        return ovl_tuning(self.ctx)

    def tuning_sap(self):
        return ovl_tuning_sap(self.ctx)

    def tuning_mrhs(self):
        return ovl_tuning_mrhs(self.ctx)

    def deflation_info(self):
        return ovl_deflation_info(self.ctx)

    def krylov_sign_info(self):
        return ovl_krylov_sign_info(self.ctx)

    def dslash_time(self, precision, reps=20):
        return ovl_dslash_time(self.ctx, precision, reps)

    def dslash_time_n(self, precision, nrhs, reps=20):
        return ovl_dslash_time_n(self.ctx, precision, nrhs, reps)

    def wilson_apply_n(self, out, inp, n_rhs, m0):
        return wilson_apply_n(self.ctx, out, inp, n_rhs, m0)

    def ovl_apply_n(self, out, inp, n_rhs, tol):
        return ovl_apply_n(self.ctx, out, inp, n_rhs, tol)

    def prof_enable(self, on=True):
        ovl_prof_enable(self.ctx, on)

    def prof_get(self, reset=False):
        return ovl_prof_get(self.ctx, reset)


class Server:
    """The library's serving loop (ovl_server_*): submit overlap solves as they arrive.

    Buffers passed to submit() must stay alive until the request is done; the object
    keeps references to them for that reason."""

    def __init__(self, slots=2, hbm_budget=0):
        self.h = ctypes.c_void_p()
        _check(lib().ovl_server_create(ctypes.byref(self.h), int(slots), int(hbm_budget)))
        self._keep = {}

    def submit(self, gauge, dims, rho, mu, b, x, n_rhs=1, tol=0.0, params=None, gauge_key=0):
        req = ovl_request()
        req.gauge = _ptr(gauge).value
        req.gauge_key = int(gauge_key)
        for m in range(4):
            req.dims[m] = int(dims[m])
        req.rho, req.mu, req.n_rhs, req.tol = float(rho), float(mu), int(n_rhs), float(tol)
        req.b = _ptr(b).value
        req.x = _ptr(x, True).value
        req.params = ctypes.cast(ctypes.byref(params), ctypes.c_void_p).value if params is not None else None
        t = ctypes.c_long()
        _check(lib().ovl_server_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (gauge, b, x, params)
        return t.value

    def query(self, ticket):
        r = ovl_result()
        _check(lib().ovl_server_query(self.h, ctypes.c_long(ticket), ctypes.byref(r)))
        return r.as_dict()

    def wait(self, ticket):
        r = ovl_result()
        _check(lib().ovl_server_wait(self.h, ctypes.c_long(ticket), ctypes.byref(r)))
        self._keep.pop(ticket, None)
        return r.as_dict()

    def report(self):
        p50, p99, sps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        hw, done, failed = ctypes.c_size_t(), ctypes.c_long(), ctypes.c_long()
        _check(lib().ovl_server_report(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(sps),
                                       ctypes.byref(hw), ctypes.byref(done), ctypes.byref(failed)))
        return {"p50_s": p50.value, "p99_s": p99.value, "solves_per_s": sps.value, "hbm_high_water": hw.value,
                "completed": done.value, "failed": failed.value}

    def close(self):
        if self.h:
            _check(lib().ovl_server_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

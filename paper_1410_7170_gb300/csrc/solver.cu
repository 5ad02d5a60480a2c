// Krylov solvers for D_N psi = eta (Eq. linsys): restarted right-preconditioned
// FGMRES(m) (GMRES(m) when no preconditioner is used), Sec. 5.1, with
//   * classical Gram-Schmidt with one re-orthogonalisation (CGS2) on the device,
//     Givens rotations of the (m+1) x m Hessenberg matrix on the host;
//   * relaxation of the sign-function accuracy eps_sign = eps/||r_k||_rel * 1e-2 (Sec. 5.2);
//   * preconditioners: an inexact Wilson solve D_W(m0_prec)^{-1} to eps_prec (Sec. 5.1,
//     with m0_prec = m0^def of Eq. default_m), or the recursive scheme of Sec. 5.3: an
//     inner FGMRES on D_N with a low-accuracy FP32 sign, itself preconditioned by the
//     Wilson solve.
// The same template runs in FP64 (outer) and FP32 (inner, Wilson) on even-odd spinors
// viewed as flat arrays of reals.
#include <math.h>
#include <string.h>

#include <chrono>
#include <complex>
#include <vector>

#include "sap.h"
#include "solver.h"

namespace ovl {

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            cudaGetLastError();                                                    \
            c->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #expr; \
            return OVL_ECUDA;                                                      \
        }                                                                          \
    } while (0)
#define ST(expr)                     \
    do {                             \
        ovl_status s_ = (expr);      \
        if (s_ != OVL_OK) return s_; \
    } while (0)

using cd = std::complex<double>;

template <typename T> struct Ops;
template <> struct Ops<double> {
    using S = double2;
    static cudaError_t norm2(Ctx *c, const double *x, double *res) { return dev_norm2(x, c->n64, res, c->rs, c->stream); }
    static cudaError_t axpby(Ctx *c, double a, const double *x, double b, double *y) {
        return dev_axpby(a, x, b, y, c->n64, c->stream);
    }
    static cudaError_t multidot(Ctx *c, const double *base, int m, const double *w, double *out) {
        return dev_multidot(base, c->n64, m, w, c->n64, out, c->d_md_part, c->stream);
    }
    static cudaError_t multiaxpy(Ctx *c, const double *base, int m, const double *coef, double *w) {
        return dev_multiaxpy(base, c->n64, m, coef, w, c->n64, c->stream);
    }
    static cudaError_t wilson(Ctx *c, const double *in, double *out, double m0) {
        return wilson_f64(c->g, c->U64, (const double2 *)in, (double2 *)out, m0, 0, 1.0, nullptr, 0.0, c->stream);
    }
    static cudaError_t sap(Ctx *c, const SapGeom &sg, const double *v, double *x, double *r, double m0) {
        return sap_f64(c->g, sg, c->U64, (const double2 *)v, (double2 *)x, (double2 *)r, m0, c->p.sap_cycles,
                       c->p.sap_mr_iters, c->stream);
    }
    static constexpr bool kCgs2 = true;
};
template <> struct Ops<float> {
    using S = float4;
    static cudaError_t norm2(Ctx *c, const float *x, double *res) { return dev_norm2_f(x, c->n64, res, c->rs, c->stream); }
    static cudaError_t axpby(Ctx *c, double a, const float *x, double b, float *y) {
        return dev_axpby_f((float)a, x, (float)b, y, c->n64, c->stream);
    }
    static cudaError_t multidot(Ctx *c, const float *base, int m, const float *w, double *out) {
        return dev_multidot_f(base, c->n64, m, w, c->n64, out, c->d_md_part, c->stream);
    }
    static cudaError_t multiaxpy(Ctx *c, const float *base, int m, const double *coef, float *w) {
        return dev_multiaxpy_f(base, c->n64, m, coef, w, c->n64, c->stream);
    }
    static cudaError_t wilson(Ctx *c, const float *in, float *out, double m0) {
        return wilson_f32(c->g, c->U32, (const float4 *)in, (float4 *)out, (float)m0, 0, 1.f, nullptr, 0.f,
                          c->stream);
    }
    static cudaError_t sap(Ctx *c, const SapGeom &sg, const float *v, float *x, float *r, double m0) {
        return sap_f32(c->g, sg, c->U32, (const float4 *)v, (float4 *)x, (float4 *)r, (float)m0, c->p.sap_cycles,
                       c->p.sap_mr_iters, c->stream);
    }
    static constexpr bool kCgs2 = false;   // low-accuracy solves: one Gram-Schmidt pass unless it cancels
};

template <typename T>
static ovl_status ensure_krylov(Ctx *c, Krylov<T> &k, int m, bool flexible) {
    if (k.V && k.m == m && k.flexible == flexible) return OVL_OK;
    if (k.V) {   // different shape requested: keep the old block (owned by ctx), take a new one
        k = Krylov<T>();
    }
    const long n = c->n64;
    const int nvec = (m + 1) + (flexible ? m : 0) + 2;
    void *buf;
    ST(c->alloc(&buf, (size_t)n * sizeof(T) * nvec));
    T *b = (T *)buf;
    k.V = b;
    k.Z = flexible ? b + (long)(m + 1) * n : nullptr;
    k.w = b + (long)((m + 1) + (flexible ? m : 0)) * n;
    k.r = k.w + n;
    k.m = m;
    k.flexible = flexible;
    return OVL_OK;
}

struct KrylovResult {
    int iters = 0;
    double rel_res = 1.0;   // last residual estimate (true residual at exit of a cycle)
    bool converged = false;
};

// Upload complex coefficients (interleaved) to the device coefficient buffer.
static ovl_status upload_coef(Ctx *c, const std::vector<cd> &v) {
    double *h = c->h_scal + 256;
    for (size_t k = 0; k < v.size(); k++) {
        h[2 * k] = v[k].real();
        h[2 * k + 1] = v[k].imag();
    }
    CK(cudaMemcpyAsync(c->d_coef, h, v.size() * 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return OVL_OK;
}

// FGMRES(m). matvec(in, out, rel_res_now) computes out = A in; precond(in, out) gives
// out ~ A^{-1} in (nullptr: plain GMRES). x holds the initial guess (x_zero: it is 0).
// Stops when ||b - A x|| <= tol ||b|| (checked on the recomputed residual) or after
// maxit iterations.
// verify = false (preconditioner solves): return after the cycle whose Arnoldi residual
// estimate meets tol, without recomputing the true residual.
template <typename T, typename MV, typename PC>
static ovl_status fgmres(Ctx *c, Krylov<T> &k, T *x, const T *b, double tol, int maxit, bool x_zero, MV matvec,
                         PC *precond, KrylovResult *res, bool verify = true) {
    using O = Ops<T>;
    const long n = c->n64;
    const int m = k.m;
    double bb;
    CK(O::norm2(c, b, c->d_scal));
    ST(c->fetch(c->d_scal, 1, &bb));
    const double bnorm = sqrt(bb);
    res->iters = 0;
    res->converged = false;
    if (bnorm == 0.0) {
        CK(cudaMemsetAsync(x, 0, n * sizeof(T), c->stream));
        res->rel_res = 0.0;
        res->converged = true;
        return OVL_OK;
    }
    bool xz = x_zero;
    if (xz) CK(cudaMemsetAsync(x, 0, n * sizeof(T), c->stream));   // x_zero: start from x = 0
    std::vector<cd> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m), h1(m + 1), h2(m + 1);
    while (true) {
        // r = b - A x
        if (xz) {
            CK(cudaMemcpyAsync(k.r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
        } else {
            ST(matvec(x, k.w, -1.0));
            CK(cudaMemcpyAsync(k.r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
            CK(O::axpby(c, -1.0, k.w, 1.0, k.r));
        }
        double rr;
        CK(O::norm2(c, k.r, c->d_scal));
        ST(c->fetch(c->d_scal, 1, &rr));
        const double beta = sqrt(rr);
        res->rel_res = beta / bnorm;
        if (!std::isfinite(beta)) {
            c->err = "Krylov solver: non-finite residual";
            return OVL_EBREAKDOWN;
        }
        if (beta <= tol * bnorm) {
            res->converged = true;
            return OVL_OK;
        }
        if (res->iters >= maxit) return OVL_OK;
        CK(O::axpby(c, 1.0 / beta, k.r, 0.0, k.V));
        std::fill(gv.begin(), gv.end(), cd(0));
        gv[0] = beta;
        int j = 0;
        bool stop = false;
        for (; j < m && !stop; j++) {
            T *vj = k.V + (long)j * n;
            T *zj = vj;
            if (precond) {
                zj = k.Z + (long)j * n;
                ST((*precond)(vj, zj));
            }
            const double rel_now = std::abs(gv[j]) / bnorm;
            ST(matvec(zj, k.w, rel_now));
            // Gram-Schmidt: h = V^H w and ||w||^2 in one round trip; a second pass (CGS2)
            // always in FP64, and in FP32 only when the first pass cancels most of w.
            double hn = 0.0;
            for (int pass = 0; pass < 2; pass++) {
                std::vector<cd> &hh = pass == 0 ? h1 : h2;
                CK(O::multidot(c, k.V, j + 1, k.w, c->d_scal));
                CK(O::norm2(c, k.w, c->d_scal + 2 * (j + 1)));
                double tmp[2 * 128 + 2];
                ST(c->fetch(c->d_scal, 2 * (j + 1) + 1, tmp));
                std::vector<cd> neg(j + 1);
                double hsq = 0.0;
                for (int i = 0; i <= j; i++) {
                    hh[i] = cd(tmp[2 * i], tmp[2 * i + 1]);
                    neg[i] = -hh[i];
                    hsq += std::norm(hh[i]);
                }
                ST(upload_coef(c, neg));
                CK(O::multiaxpy(c, k.V, j + 1, c->d_coef, k.w));
                const double ww = tmp[2 * (j + 1)];
                const double left = ww - hsq;   // ||w - V h||^2 for orthonormal V
                if (pass == 0 && !O::kCgs2 && left > 0.1 * ww) {
                    std::fill(h2.begin(), h2.end(), cd(0));
                    hn = sqrt(left);
                    break;
                }
                if (pass == 1) {
                    double w2;
                    CK(O::norm2(c, k.w, c->d_scal));
                    ST(c->fetch(c->d_scal, 1, &w2));
                    hn = sqrt(w2);
                }
            }
            for (int i = 0; i <= j; i++) H[(size_t)i * m + j] = h1[i] + h2[i];
            H[(size_t)(j + 1) * m + j] = hn;
            if (!std::isfinite(hn)) {
                c->err = "Krylov solver: non-finite Arnoldi coefficient";
                return OVL_EBREAKDOWN;
            }
            if (hn > 0) CK(O::axpby(c, 1.0 / hn, k.w, 0.0, k.V + (long)(j + 1) * n));
            // rotations
            for (int i = 0; i < j; i++) {
                const cd a = H[(size_t)i * m + j], bq = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bq;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bq;
            }
            const cd a = H[(size_t)j * m + j], bq = H[(size_t)(j + 1) * m + j];
            const double den = sqrt(std::norm(a) + std::norm(bq));
            cs[j] = den > 0 ? a / den : cd(1.0);
            sn[j] = den > 0 ? bq / den : cd(0.0);
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = std::conj(cs[j]) * gv[j];
            res->iters++;
            if (std::abs(gv[j + 1]) <= tol * bnorm || hn == 0.0 || res->iters >= maxit) stop = true;
        }
        // y = H^{-1} g, x += Z y
        for (int i = j - 1; i >= 0; i--) {
            cd s = gv[i];
            for (int q = i + 1; q < j; q++) s -= H[(size_t)i * m + q] * y[q];
            y[i] = s / H[(size_t)i * m + i];
        }
        std::vector<cd> yy(y.begin(), y.begin() + j);
        ST(upload_coef(c, yy));
        CK(O::multiaxpy(c, precond ? k.Z : k.V, j, c->d_coef, x));
        xz = false;
        if (!verify && (std::abs(gv[j]) <= tol * bnorm || res->iters >= maxit)) {
            res->rel_res = std::abs(gv[j]) / bnorm;
            res->converged = res->rel_res <= tol;
            return OVL_OK;
        }
    }
}

// ------------------------------------------------------------------ preconditioners
// Inexact Wilson solve out ~ D_W(m0_prec)^{-1} in to eps_prec (Sec. 5.1), precision T:
// FGMRES(prec_restart) on D_W(m0_prec), right-preconditioned by SAP cycles.
template <typename T>
static ovl_status wilson_solve(Ctx *c, Krylov<T> &k, const T *in, T *out, double m0, double tol, int *iters = nullptr) {
    ST(ensure_krylov<T>(c, k, c->p.prec_restart, true));
    T *&scratch = sizeof(T) == 8 ? (T *&)c->sap_r64 : (T *&)c->sap_r32;
    if (!scratch) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(T)));
        scratch = (T *)buf;
    }
    const SapGeom sg = make_sap_geom(c->g, c->p.sap_block);
    auto mv = [&](const T *a, T *o, double) -> ovl_status {
        CK(Ops<T>::wilson(c, a, o, m0));
        return OVL_OK;
    };
    auto pc = [&](const T *a, T *o) -> ovl_status {
        CK(Ops<T>::sap(c, sg, a, o, scratch, m0));
        return OVL_OK;
    };
    KrylovResult r;
    ST(fgmres<T>(c, k, out, in, tol, c->p.prec_max_iter, true, mv, &pc, &r, false));
    c->stat_prec += r.iters;
    if (iters) *iters = r.iters;
    return OVL_OK;
}

static double relax_tol(Ctx *c, double target, double rel_now, double lo, double hi) {
    if (!c->p.relax || rel_now <= 0) return lo;
    double e = target / rel_now * c->p.relax_factor;
    return std::min(hi, std::max(lo, e));
}

// Inner FP32 FGMRES on D_N (Sec. 5.3): low-accuracy FP32 sign, Wilson preconditioner.
static ovl_status inner_solve(Ctx *c, const float *in, float *out) {
    ST(ensure_krylov<float>(c, c->kry_inner, c->p.restart_inner, true));
    const double eps = c->p.eps_inner;
    auto mv = [&](const float *a, float *o, double rel_now) -> ovl_status {
        const double t = relax_tol(c, eps, rel_now < 0 ? eps : rel_now, 1e-6, 1e-1);
        return c->sign32((const float4 *)a, (float4 *)o, t, 1);
    };
    auto pc = [&](const float *a, float *o) -> ovl_status {
        return wilson_solve<float>(c, c->kry_wil32, a, o, c->m0_prec, c->p.eps_prec);
    };
    KrylovResult r;
    ST(fgmres<float>(c, c->kry_inner, out, in, eps, c->p.max_inner, true, mv, &pc, &r, false));
    c->stat_inner += r.iters;
    return OVL_OK;
}

static ovl_status ensure_f32_buffers(Ctx *c) {
    if (!c->f_a) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(float) * 2));
        c->f_a = (float *)buf;
        c->f_b = c->f_a + c->n64;
    }
    return OVL_OK;
}

// Right preconditioner of the outer FP64 FGMRES: z ~ M^{-1} v.
static ovl_status outer_precond(Ctx *c, const double *v, double *z) {
    const bool mixed = c->p.precision != OVL_FP64 || c->p.precond == OVL_PREC_RECURSIVE;
    if (!mixed && c->p.precond == OVL_PREC_WILSON)
        return wilson_solve<double>(c, c->kry_wil64, v, z, c->m0_prec, c->p.eps_prec);
    ST(ensure_f32_buffers(c));
    CK(spinor_d2f(c->g, (const double2 *)v, (float4 *)c->f_a, c->stream));
    if (c->p.precond == OVL_PREC_WILSON) ST(wilson_solve<float>(c, c->kry_wil32, c->f_a, c->f_b, c->m0_prec, c->p.eps_prec));
    else ST(inner_solve(c, c->f_a, c->f_b));
    CK(spinor_f2d(c->g, (const float4 *)c->f_b, (double2 *)z, c->stream));
    return OVL_OK;
}

ovl_status wilson_solve_eo(Ctx *c, const double2 *b, double2 *x, double m0, double tol, int *iters) {
    if (c->p.precision == OVL_FP64) return wilson_solve<double>(c, c->kry_wil64, (const double *)b, (double *)x, m0, tol, iters);
    ST(ensure_f32_buffers(c));
    CK(spinor_d2f(c->g, b, (float4 *)c->f_a, c->stream));
    ST(wilson_solve<float>(c, c->kry_wil32, c->f_a, c->f_b, m0, tol, iters));
    CK(spinor_f2d(c->g, (const float4 *)c->f_b, x, c->stream));
    return OVL_OK;
}

ovl_status solve_all(Ctx *c, double *x, const double *b, int n_rhs, double tol, ovl_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    c->stat_ms64 = c->stat_ms32 = c->stat_prec = 0;
    c->stat_inner = 0;
    const bool flexible = c->p.precond != OVL_PREC_NONE;
    ST(ensure_krylov<double>(c, c->kry_outer, c->p.restart, flexible));
    if (!c->d_x) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2));
        c->d_x = (double2 *)buf;
        c->d_b = c->d_x + c->g.V * 12;
    }
    int outer_total = 0;
    double worst = 0.0;
    bool all_conv = true;
    const double tight = std::max(1e-14, std::min(c->p.sign_tol, 0.1 * tol));
    for (int r = 0; r < n_rhs; r++) {
        const double *br = b + (size_t)r * c->n64;
        double *xr = x + (size_t)r * c->n64;
        ST(c->import_vec(br, c->d_b));
        ST(c->import_vec(xr, c->d_x));
        double xx;
        ST(c->norm2_d((const double *)c->d_x, &xx));
        // D_N in FP64; in the mixed modes, a relaxed product whose requested accuracy is
        // within reach of the lower-precision multishift (Sec. 5.2 lets it grow as the
        // residual falls) runs in FP32 (FP16-stored directions in OVL_MIXED_HALF).
        const bool mixed = c->p.precision != OVL_FP64;
        const double low_ok = c->p.precision == OVL_MIXED_HALF ? 1e-3 : 1e-5;
        auto mv = [&](const double *a, double *o, double rel_now) -> ovl_status {
            const double t = rel_now < 0 ? tight : relax_tol(c, tol, rel_now, tight, 1e-1);
            if (mixed && rel_now >= 0 && t >= low_ok) {
                ST(ensure_f32_buffers(c));
                CK(spinor_d2f(c->g, (const double2 *)a, (float4 *)c->f_a, c->stream));
                ST(c->sign32((const float4 *)c->f_a, (float4 *)c->f_b, t, 1));
                CK(spinor_f2d(c->g, (const float4 *)c->f_b, (double2 *)o, c->stream));
                return OVL_OK;
            }
            return c->sign64((const double2 *)a, (double2 *)o, t, 1);
        };
        auto pc = [&](const double *a, double *o) -> ovl_status { return outer_precond(c, a, o); };
        KrylovResult kr;
        ovl_status s;
        if (flexible) s = fgmres<double>(c, c->kry_outer, (double *)c->d_x, (const double *)c->d_b, tol,
                                         c->p.max_iter, xx == 0.0, mv, &pc, &kr);
        else {
            using NoPC = ovl_status (*)(const double *, double *);
            s = fgmres<double>(c, c->kry_outer, (double *)c->d_x, (const double *)c->d_b, tol, c->p.max_iter,
                               xx == 0.0, mv, (NoPC *)nullptr, &kr);
        }
        if (s != OVL_OK) return s;
        outer_total += kr.iters;
        worst = std::max(worst, kr.rel_res);
        all_conv = all_conv && kr.converged;
        ST(c->export_vec(c->d_x, xr));
    }
    if (stats) {
        stats->outer_iters = outer_total;
        stats->inner_iters = c->stat_inner;
        stats->ms_iters_fp64 = c->stat_ms64;
        stats->ms_iters_low = c->stat_ms32;
        stats->prec_iters = c->stat_prec;
        stats->true_rel_resid = worst;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!all_conv) {
        c->err = "ovl_solve: tolerance not reached within max_iter";
        return OVL_ENOCONV;
    }
    return OVL_OK;
}

}  // namespace ovl

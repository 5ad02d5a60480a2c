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

#include <algorithm>
#include <chrono>
#include <complex>
#include <memory>
#include <vector>

#include "sap.h"
#include "solver.h"

namespace ovl {

using cd = std::complex<double>;

template <typename T> struct Ops;
template <> struct Ops<double> {
    using S = double2;
    static cudaError_t norm2(Ctx *c, const double *x, double *res) { return dev_norm2(x, c->n64, res, c->rs, c->stream); }
    static cudaError_t axpby(Ctx *c, double a, const double *x, double b, double *y) {
        return dev_axpby(a, x, b, y, c->n64, c->stream);
    }
    // basis vectors k = 0..m-1 at base + k * stride (stride 0: consecutive vectors)
    static cudaError_t multidot(Ctx *c, const double *base, int m, const double *w, double *out, long stride = 0) {
        return dev_multidot(base, stride ? stride : c->n64, m, w, c->n64, out, c->d_md_part, c->stream);
    }
    static cudaError_t multiaxpy(Ctx *c, const double *base, int m, const double *coef, double *w, long stride = 0) {
        return dev_multiaxpy(base, stride ? stride : c->n64, m, coef, w, c->n64, c->stream);
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
    static cudaError_t multidot(Ctx *c, const float *base, int m, const float *w, double *out, long stride = 0) {
        return dev_multidot_f(base, stride ? stride : c->n64, m, w, c->n64, out, c->d_md_part, c->stream);
    }
    static cudaError_t multiaxpy(Ctx *c, const float *base, int m, const double *coef, float *w, long stride = 0) {
        return dev_multiaxpy_f(base, stride ? stride : c->n64, m, coef, w, c->n64, c->stream);
    }
    static cudaError_t wilson(Ctx *c, const float *in, float *out, double m0) {
        return wilson_f32(c->g, c->U32, (const float4 *)in, (float4 *)out, (float)m0, 0, 1.f, nullptr, 0.f,
                          c->stream);
    }
    static cudaError_t sap(Ctx *c, const SapGeom &sg, const float *v, float *x, float *r, double m0) {
        return sap_f32(c->g, sg, c->U32, (const float4 *)v, (float4 *)x, (float4 *)r, (float)m0, c->p.sap_cycles,
                       c->p.sap_mr_iters, c->stream);
    }
    // [0, 2m) = <base_j, w>, [2m] = ||w||^2 in one pass over the basis
    static cudaError_t multidot_norm(Ctx *c, const float *base, int m, const float *w, double *out) {
        return dev_multidot_norm_f(base, c->n64, m, w, c->n64, out, c->d_md_part, c->stream);
    }
    // out = scale (w - sum_j h_j base_j), h on the device
    static cudaError_t orth_scale(Ctx *c, const float *base, int m, const double *h, double scale, const float *w,
                                  float *out) {
        return dev_orth_scale_f(base, c->n64, m, h, scale, w, out, c->n64, c->stream);
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

ovl_status upload_coef(Ctx *c, const std::vector<cd> &v) {
    double *h = c->h_scal + kScal / 2;
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
                c->fgmres_rel = std::abs(gv[j]) / bnorm;   // read by an adaptive preconditioner
                ST((*precond)(vj, zj));
            }
            const double rel_now = std::abs(gv[j]) / bnorm;
            ST(matvec(zj, k.w, rel_now));
            // Gram-Schmidt: h = V^H w and ||w||^2 in one round trip; a second pass (CGS2)
            // always in FP64, and in FP32 only when the first pass cancels most of w.
            double hn = 0.0;
            bool next_done = false;   // V_{j+1} already written
            if constexpr (!O::kCgs2) {
                // one pass: the dots and ||w||^2 in one kernel; unless the pass cancels most of w,
                // V_{j+1} = (w - V h) / hn in one more, with h read from device memory
                CK(O::multidot_norm(c, k.V, j + 1, k.w, c->d_scal));
                double tmp[2 * 128 + 2];
                ST(c->fetch(c->d_scal, 2 * (j + 1) + 1, tmp));
                double hsq = 0.0;
                for (int i = 0; i <= j; i++) {
                    h1[i] = cd(tmp[2 * i], tmp[2 * i + 1]);
                    hsq += std::norm(h1[i]);
                }
                const double ww = tmp[2 * (j + 1)];
                const double left = ww - hsq;
                if (left > 0.1 * ww) {
                    std::fill(h2.begin(), h2.end(), cd(0));
                    hn = sqrt(left);
                    if (hn > 0) CK(O::orth_scale(c, k.V, j + 1, c->d_scal, 1.0 / hn, k.w, k.V + (long)(j + 1) * n));
                    next_done = true;
                } else {   // cancellation: subtract this pass, then a second full pass below
                    std::vector<cd> neg(j + 1);
                    for (int i = 0; i <= j; i++) neg[i] = -h1[i];
                    ST(upload_coef(c, neg));
                    CK(O::multiaxpy(c, k.V, j + 1, c->d_coef, k.w));
                }
            }
            for (int pass = next_done ? 2 : (O::kCgs2 ? 0 : 1); pass < 2; pass++) {
                std::vector<cd> &hh = pass == 0 ? h1 : h2;
                CK(O::multidot(c, k.V, j + 1, k.w, c->d_scal));
                CK(O::norm2(c, k.w, c->d_scal + 2 * (j + 1)));
                double tmp[2 * 128 + 2];
                ST(c->fetch(c->d_scal, 2 * (j + 1) + 1, tmp));   // 2 (j + 1) + 1 <= 243 doubles
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
            if (hn > 0 && !next_done) CK(O::axpby(c, 1.0 / hn, k.w, 0.0, k.V + (long)(j + 1) * n));
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
    PhaseClock pclk(c, &c->t_prec);
    ST(ensure_krylov<T>(c, k, c->p.prec_restart, true));
    T *&scratch = sizeof(T) == 8 ? (T *&)c->sap_r64 : (T *&)c->sap_r32;
    if (!scratch) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(T)));
        scratch = (T *)buf;
    }
    SapGeom sg = make_sap_geom(c->g, c->p.sap_block);
    sg.tps = c->sap_tps;
    auto mv = [&](const T *a, T *o, double) -> ovl_status {
        CK(Ops<T>::wilson(c, a, o, m0));
        return OVL_OK;
    };
    auto pc = [&](const T *a, T *o) -> ovl_status {
        if (sizeof(T) == 4 && c->p.wilson_mg) return mg_apply_f32(c, (const float4 *)a, (float4 *)o, m0);
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

// Wilson preconditioner mass for the next inner FGMRES iteration (params.m0_adapt), Sec. 5.1:
// the paper observes that the best m0_prec is not known a priori and suggests approximating
// it "on the fly" by changing it from one preconditioned FGMRES iteration to the next, without
// a rule. Reading: five candidates spread evenly over [1.5 m0_def, 0] (the part of the paper's
// scan range [-sigma~_min, 0] around m0_def; 0 included); the application made
// with candidate i is credited, once the next iteration starts, with the drop of the FGMRES
// residual estimate, -log(r_new / r_old), and with the wall time in between (its Wilson solve
// and the D_N product of that iteration). Each candidate is tried twice, then the one with the
// largest credited drop per second is used, with a random candidate one time in eight.
static double m0_adapt_pick(Ctx *c, double rel_now) {
    Ctx::M0Adapt &a = c->m0a;
    const auto now = std::chrono::steady_clock::now();
    if (a.cand.empty()) {
        const double m = c->m0_prec;
        for (int k = 0; k < 5; k++) a.cand.push_back(m * (1.5 - 0.375 * k));
        a.gain.assign(5, 0.0);
        a.cost.assign(5, 0.0);
        a.n.assign(5, 0);
    }
    if (a.pending >= 0 && rel_now > 0 && a.rel_pending > 0) {
        a.gain[a.pending] += std::max(0.0, -log(rel_now / a.rel_pending));
        a.cost[a.pending] += std::chrono::duration<double>(now - a.t_pending).count();
        a.n[a.pending]++;
    }
    const int K = (int)a.cand.size();
    int pick = -1;
    for (int k = 0; k < K && pick < 0; k++)
        if (a.n[k] < 2) pick = k;
    if (pick < 0) {
        a.rng ^= a.rng << 13;
        a.rng ^= a.rng >> 7;
        a.rng ^= a.rng << 17;
        if (a.rng % 8 == 0) {
            pick = (int)((a.rng >> 8) % K);
        } else {
            double best = -1.0;
            for (int k = 0; k < K; k++) {
                const double e = a.cost[k] > 0 ? a.gain[k] / a.cost[k] : 0.0;
                if (e > best) {
                    best = e;
                    pick = k;
                }
            }
        }
    }
    a.pending = pick;
    a.rel_pending = rel_now;
    a.t_pending = now;
    a.uses++;
    return a.cand[pick];
}

// Inner FP32 FGMRES on D_N (Sec. 5.3): low-accuracy FP32 sign, Wilson preconditioner.
static ovl_status inner_solve(Ctx *c, const float *in, float *out) {
    ST(ensure_krylov<float>(c, c->kry_inner, c->p.restart_inner, true));
    const double eps = c->p.eps_inner;
    auto mv = [&](const float *a, float *o, double rel_now) -> ovl_status {
        const double t = relax_tol(c, eps, rel_now < 0 ? eps : rel_now, 1e-6, 1e-1);
        return c->sign32((const float4 *)a, (float4 *)o, t, 1);
    };
    c->m0a.pending = -1;   // a new inner solve: nothing to credit from the previous one
    auto pc = [&](const float *a, float *o) -> ovl_status {
        const double m0 = c->p.m0_adapt ? m0_adapt_pick(c, c->fgmres_rel) : c->m0_prec;
        return wilson_solve<float>(c, c->kry_wil32, a, o, m0, c->p.eps_prec);
    };
    KrylovResult r;
    ST(fgmres<float>(c, c->kry_inner, out, in, eps, c->p.max_inner, true, mv, &pc, &r, false));
    c->stat_inner += r.iters;
    return OVL_OK;
}

ovl_status ensure_f32_buffers(Ctx *c) {
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

// One application of the Schwarz preconditioner, x = M_SAP b: params.sap_cycles red-black
// cycles from x = 0 over params.sap_block blocks, params.sap_mr_iters MR steps per block
// solve, on D_W(m0); FP64 even-odd spinors in and out, FP32 inside unless precision ==
// OVL_FP64. The same call the Wilson FGMRES makes for its preconditioner.
ovl_status sap_apply_eo(Ctx *c, const double2 *b, double2 *x, double m0) {
    SapGeom sg = make_sap_geom(c->g, c->p.sap_block);
    sg.tps = c->sap_tps;
    if (c->p.precision == OVL_FP64) {
        if (!c->sap_r64) {
            void *buf;
            ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double)));
            c->sap_r64 = buf;
        }
        CK(Ops<double>::sap(c, sg, (const double *)b, (double *)x, (double *)c->sap_r64, m0));
        return OVL_OK;
    }
    ST(ensure_f32_buffers(c));
    if (!c->sap_r32) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(float)));
        c->sap_r32 = buf;
    }
    CK(spinor_d2f(c->g, b, (float4 *)c->f_a, c->stream));
    CK(Ops<float>::sap(c, sg, c->f_a, c->f_b, (float *)c->sap_r32, m0));
    CK(spinor_f2d(c->g, (const float4 *)c->f_b, x, c->stream));
    return OVL_OK;
}

int batch_size_for(Ctx *c, int want);
// Most accurate sign request the lower-precision multishift serves in the mixed modes:
// FP32 vectors (the accuracy floor of the inner requests too), FP16-stored directions (11
// significant bits, per-site scale), BF16-stored directions (8 significant bits).
static double low_sign_floor(int precision) {
    return precision == OVL_MIXED_BF16 ? 1e-2 : precision == OVL_MIXED_HALF ? 1e-3 : 1e-6;
}


// The wall-clock limit of a solve (params.max_seconds), armed for the duration of one call.
struct DeadlineScope {
    Ctx *c;
    DeadlineScope(Ctx *c_, std::chrono::steady_clock::time_point t0) : c(c_) {
        c->has_deadline = c->p.max_seconds > 0;
        if (c->has_deadline)
            c->deadline = t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                   std::chrono::duration<double>(c->p.max_seconds));
    }
    ~DeadlineScope() { c->has_deadline = false; }
};

ovl_status solve_all(Ctx *c, double *x, const double *b, int n_rhs, double tol, ovl_stats *stats) {
    const auto t0 = std::chrono::steady_clock::now();
    DeadlineScope dl(c, t0);
    c->stat_ms64 = c->stat_ms32 = c->stat_msff = c->stat_prec = 0;
    c->stat_inner = 0;
    c->t_sign64 = c->t_sign_low = c->t_prec = 0;
    const bool flexible = c->p.precond != OVL_PREC_NONE;
    int outer_total = 0;
    double worst = 0.0;
    bool all_conv = true;
    const double tight = std::max(1e-14, std::min(c->p.sign_tol, 0.1 * tol));
    if (n_rhs > 1 && c->p.rhs_block > 1) {
        // several right-hand sides in lock-step batches sized to the free device memory
        const int nbmax = batch_size_for(c, std::min(c->p.rhs_block, n_rhs));
        if (!c->xbat || c->xbat_cap < nbmax) {
            void *buf;
            ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2 * nbmax));
            c->xbat = (double2 *)buf;
            c->bbat = c->xbat + (size_t)nbmax * c->g.V * 12;
            c->xbat_cap = nbmax;
        }
        for (int r0 = 0; r0 < n_rhs; r0 += nbmax) {
            const int nb = std::min(nbmax, n_rhs - r0);
            for (int y = 0; y < nb; y++) {
                ST(c->import_vec(b + (size_t)(r0 + y) * c->n64, c->bbat + (size_t)y * c->g.V * 12));
                ST(c->import_vec(x + (size_t)(r0 + y) * c->n64, c->xbat + (size_t)y * c->g.V * 12));
            }
            int its;
            double wr;
            bool cv;
            ST(solve_batch(c, c->xbat, c->bbat, nb, tol, &its, &wr, &cv));
            outer_total += its;
            worst = std::max(worst, wr);
            all_conv = all_conv && cv;
            for (int y = 0; y < nb; y++) ST(c->export_vec(c->xbat + (size_t)y * c->g.V * 12, x + (size_t)(r0 + y) * c->n64));
        }
        n_rhs = 0;   // done; fall through to the statistics
    }
    if (n_rhs > 0) {
        ST(ensure_krylov<double>(c, c->kry_outer, c->p.restart, flexible));
        if (!c->d_x) {
            void *buf;
            ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2));
            c->d_x = (double2 *)buf;
            c->d_b = c->d_x + c->g.V * 12;
        }
    }
    for (int r = 0; r < n_rhs; r++) {
        const double *br = b + (size_t)r * c->n64;
        double *xr = x + (size_t)r * c->n64;
        ST(c->import_vec(br, c->d_b));
        ST(c->import_vec(xr, c->d_x));
        double xx;
        ST(c->norm2_d((const double *)c->d_x, &xx));
        // D_N in FP64; in the mixed modes, a relaxed product whose requested accuracy is
        // within reach of the lower-precision multishift (Sec. 5.2 lets it grow as the
        // residual falls) runs in FP32 (16-bit stored directions in OVL_MIXED_HALF/BF16).
        const bool mixed = c->p.precision != OVL_FP64;
        const double low_ok = low_sign_floor(c->p.precision);
        auto mv = [&](const double *a, double *o, double rel_now) -> ovl_status {
            const double t = rel_now < 0 ? tight : relax_tol(c, tol, rel_now, tight, 1e-1);
            if (mixed && rel_now >= 0 && t >= low_ok) {
                ST(ensure_f32_buffers(c));
                CK(spinor_d2f(c->g, (const double2 *)a, (float4 *)c->f_a, c->stream));
                ST(c->sign32((const float4 *)c->f_a, (float4 *)c->f_b, t, 1));
                CK(spinor_f2d(c->g, (const float4 *)c->f_b, (double2 *)o, c->stream));
                return OVL_OK;
            }
            return c->sign_outer((const double2 *)a, (double2 *)o, t, 1);
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
        stats->ms_iters_ff = c->stat_msff;
        stats->prec_iters = c->stat_prec;
        stats->true_rel_resid = worst;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->t_sign_fp64 = c->t_sign64;
        stats->t_sign_low = c->t_sign_low;
        stats->t_prec = c->t_prec;
    }
    if (!all_conv) {
        c->err = "ovl_solve: tolerance not reached within max_iter";
        return OVL_ENOCONV;
    }
    return OVL_OK;
}

// ====================================================================================
// Several right-hand sides in lock-step.
//
// fgmres_batch runs nb independent FGMRES(m) iterations side by side: every basis entry
// holds nb vectors back to back, so the operator and the preconditioner are applied to
// all systems in one batched call (one multi-RHS stencil per application), while each
// system keeps its own Hessenberg matrix, Givens rotations, relaxation and stopping test.
// A system that has converged is dropped from the Gram-Schmidt work and its operator
// applications are skipped inside the batched calls (tolerance <= 0).
// ====================================================================================
// nb FP64 <-> FP32 internal spinors back to back
cudaError_t spinor_d2f_n(Ctx *c, const double2 *a, float4 *b, int nb) {
    for (int y = 0; y < nb; y++) {
        cudaError_t e = spinor_d2f(c->g, a + (long)y * c->g.V * 12, b + (long)y * c->g.V * 6, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t spinor_f2d_n(Ctx *c, const float4 *a, double2 *b, int nb) {
    for (int y = 0; y < nb; y++) {
        cudaError_t e = spinor_f2d(c->g, a + (long)y * c->g.V * 6, b + (long)y * c->g.V * 12, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

// Zero the input rows of systems that are not iterating, so a nested batched solve
// treats them as converged (zero right-hand side) and spends no work on them.
template <typename T>
cudaError_t zero_inactive(Ctx *c, T *in, int nb, const char *act) {
    for (int y = 0; y < nb; y++)
        if (!act[y]) {
            cudaError_t e = cudaMemsetAsync(in + (long)y * c->n64, 0, c->n64 * sizeof(T), c->stream);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

template <typename T>
ovl_status ensure_krylov_batch(Ctx *c, Krylov<T> &k, int &cap, int m, int nb) {
    if (k.V && k.m == m && cap >= nb) return OVL_OK;
    const long n = c->n64;
    const int nvec = (2 * m + 1 + 2) * nb;
    void *buf;
    ST(c->alloc(&buf, (size_t)n * sizeof(T) * nvec));
    T *b = (T *)buf;
    k.V = b;
    k.Z = b + (long)(m + 1) * nb * n;
    k.w = k.Z + (long)m * nb * n;
    k.r = k.w + (long)nb * n;
    k.m = m;
    k.flexible = true;
    cap = nb;
    return OVL_OK;
}

// matvec(in, out, rel[nb]): out_y = A in_y (rel[y] < 0: full accuracy; rel[y] = 2: skip y)
// precond(in, out, active[nb]): out_y ~ A^{-1} in_y for active y
template <typename T, typename MV, typename PC>
ovl_status fgmres_batch(Ctx *c, Krylov<T> &k, int nb, T *x, const T *b, double tol, int maxit, bool x_zero,
                        MV matvec, PC precond, int *iters, double *rel_out, bool *conv_out, bool verify) {
    using O = Ops<T>;
    const long n = c->n64;
    const int m = k.m;
    auto vec = [&](T *base, int j, int y) { return base + ((long)j * nb + y) * n; };
    std::vector<double> bnorm(nb), rel(nb), beta(nb);
    std::vector<char> active(nb, 1), conv(nb, 0);
    double tmp[2 * 128 + 2];
    for (int y = 0; y < nb; y++) {
        CK(O::norm2(c, b + (long)y * n, c->d_scal + y));
    }
    ST(c->fetch(c->d_scal, nb, tmp));
    for (int y = 0; y < nb; y++) bnorm[y] = sqrt(tmp[y]);
    if (x_zero) CK(cudaMemsetAsync(x, 0, (size_t)nb * n * sizeof(T), c->stream));
    bool xz = x_zero;
    int its = 0;
    std::vector<std::vector<cd>> H(nb), cs(nb), sn(nb), gv(nb);
    for (int y = 0; y < nb; y++) {
        H[y].assign((size_t)(m + 1) * m, cd(0));
        cs[y].assign(m, cd(0));
        sn[y].assign(m, cd(0));
        gv[y].assign(m + 1, cd(0));
        if (bnorm[y] == 0.0) {
            active[y] = 0;
            conv[y] = 1;
        }
    }
    std::vector<double> relv(nb);
    while (true) {
        // R = B - A X for the active systems
        if (xz) {
            CK(cudaMemcpyAsync(k.r, b, (size_t)nb * n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
        } else {
            for (int y = 0; y < nb; y++) relv[y] = active[y] ? -1.0 : 2.0;
            ST(matvec(x, k.w, relv.data()));
            CK(cudaMemcpyAsync(k.r, b, (size_t)nb * n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
            for (int y = 0; y < nb; y++)
                if (active[y]) CK(O::axpby(c, -1.0, k.w + (long)y * n, 1.0, k.r + (long)y * n));
        }
        for (int y = 0; y < nb; y++) CK(O::norm2(c, k.r + (long)y * n, c->d_scal + y));
        ST(c->fetch(c->d_scal, nb, tmp));
        bool any = false;
        for (int y = 0; y < nb; y++) {
            if (!active[y]) continue;
            beta[y] = sqrt(tmp[y]);
            rel[y] = beta[y] / bnorm[y];
            if (!std::isfinite(beta[y])) {
                c->err = "batched Krylov solver: non-finite residual";
                return OVL_EBREAKDOWN;
            }
            if (beta[y] <= tol * bnorm[y]) {
                active[y] = 0;
                conv[y] = 1;
            } else {
                any = true;
            }
        }
        if (!any || its >= maxit) break;
        for (int y = 0; y < nb; y++) {
            std::fill(gv[y].begin(), gv[y].end(), cd(0));
            gv[y][0] = beta[y];
            if (active[y]) CK(O::axpby(c, 1.0 / beta[y], k.r + (long)y * n, 0.0, vec(k.V, 0, y)));
            else CK(cudaMemsetAsync(vec(k.V, 0, y), 0, n * sizeof(T), c->stream));
        }
        std::vector<char> live = active;   // systems iterating in this cycle
        int j = 0;
        for (; j < m; j++) {
            bool alive = false;
            for (int y = 0; y < nb; y++) alive = alive || live[y];
            if (!alive) break;
            ST(precond(vec(k.V, j, 0), vec(k.Z, j, 0), live.data()));
            for (int y = 0; y < nb; y++) relv[y] = live[y] ? std::abs(gv[y][j]) / bnorm[y] : 2.0;
            ST(matvec(vec(k.Z, j, 0), k.w, relv.data()));
            // Gram-Schmidt per system: one pass, a second when it cancels (always in FP64)
            std::vector<std::vector<cd>> h1(nb, std::vector<cd>(j + 1)), h2(nb, std::vector<cd>(j + 1));
            std::vector<double> hn(nb, 0.0);
            std::vector<char> need2(nb, 0);
            for (int pass = 0; pass < 2; pass++) {
                int cnt = 0;
                for (int y = 0; y < nb; y++) {
                    if (!live[y] || (pass == 1 && !need2[y])) continue;
                    CK(O::multidot(c, vec(k.V, 0, y), j + 1, k.w + (long)y * n, c->d_scal + cnt * (2 * (j + 1) + 1),
                                   (long)nb * n));
                    CK(O::norm2(c, k.w + (long)y * n, c->d_scal + cnt * (2 * (j + 1) + 1) + 2 * (j + 1)));
                    cnt++;
                }
                if (!cnt) break;
                std::vector<double> all((size_t)cnt * (2 * (j + 1) + 1));
                if (all.size() > (size_t)kScal / 2) {
                    c->err = "batched Krylov solver: scalar staging too small";
                    return OVL_EINVAL;
                }
                ST(c->fetch(c->d_scal, (int)all.size(), all.data()));
                cnt = 0;
                for (int y = 0; y < nb; y++) {
                    if (!live[y] || (pass == 1 && !need2[y])) continue;
                    const double *t = all.data() + (size_t)cnt * (2 * (j + 1) + 1);
                    std::vector<cd> &hh = pass == 0 ? h1[y] : h2[y];
                    std::vector<cd> neg(j + 1);
                    double hsq = 0.0;
                    for (int i = 0; i <= j; i++) {
                        hh[i] = cd(t[2 * i], t[2 * i + 1]);
                        neg[i] = -hh[i];
                        hsq += std::norm(hh[i]);
                    }
                    ST(upload_coef(c, neg));
                    CK(O::multiaxpy(c, vec(k.V, 0, y), j + 1, c->d_coef, k.w + (long)y * n, (long)nb * n));
                    ST(c->sync());   // the coefficient staging is reused by the next system
                    const double ww = t[2 * (j + 1)];
                    const double left = ww - hsq;
                    if (pass == 0) {
                        if (!O::kCgs2 && left > 0.1 * ww) hn[y] = sqrt(left);
                        else need2[y] = 1;
                    } else {
                        hn[y] = sqrt(std::max(0.0, left));
                    }
                    cnt++;
                }
            }
            for (int y = 0; y < nb; y++) {
                if (!live[y]) continue;
                std::vector<cd> &Hy = H[y];
                for (int i = 0; i <= j; i++) Hy[(size_t)i * m + j] = h1[y][i] + (need2[y] ? h2[y][i] : cd(0));
                Hy[(size_t)(j + 1) * m + j] = hn[y];
                if (!std::isfinite(hn[y])) {
                    c->err = "batched Krylov solver: non-finite Arnoldi coefficient";
                    return OVL_EBREAKDOWN;
                }
                if (hn[y] > 0) CK(O::axpby(c, 1.0 / hn[y], k.w + (long)y * n, 0.0, vec(k.V, j + 1, y)));
                else CK(cudaMemsetAsync(vec(k.V, j + 1, y), 0, n * sizeof(T), c->stream));
                for (int i = 0; i < j; i++) {
                    const cd a = Hy[(size_t)i * m + j], bq = Hy[(size_t)(i + 1) * m + j];
                    Hy[(size_t)i * m + j] = std::conj(cs[y][i]) * a + std::conj(sn[y][i]) * bq;
                    Hy[(size_t)(i + 1) * m + j] = -sn[y][i] * a + cs[y][i] * bq;
                }
                const cd a = Hy[(size_t)j * m + j], bq = Hy[(size_t)(j + 1) * m + j];
                const double den = sqrt(std::norm(a) + std::norm(bq));
                cs[y][j] = den > 0 ? a / den : cd(1.0);
                sn[y][j] = den > 0 ? bq / den : cd(0.0);
                Hy[(size_t)j * m + j] = den;
                Hy[(size_t)(j + 1) * m + j] = 0.0;
                gv[y][j + 1] = -sn[y][j] * gv[y][j];
                gv[y][j] = std::conj(cs[y][j]) * gv[y][j];
                if (std::abs(gv[y][j + 1]) <= tol * bnorm[y] || hn[y] == 0.0) live[y] = 0;
            }
            its++;
            if (its >= maxit) {
                j++;
                break;
            }
        }
        // x_y += Z_y (H_y^{-1} g_y) over the columns this system took
        for (int y = 0; y < nb; y++) {
            if (!active[y]) continue;
            int jy = 0;   // columns used by y: those with nonzero diagonal
            while (jy < j && std::abs(H[y][(size_t)jy * m + jy]) > 0) jy++;
            if (!jy) continue;
            std::vector<cd> yy(jy);
            for (int i = jy - 1; i >= 0; i--) {
                cd sacc = gv[y][i];
                for (int q = i + 1; q < jy; q++) sacc -= H[y][(size_t)i * m + q] * yy[q];
                yy[i] = sacc / H[y][(size_t)i * m + i];
            }
            ST(upload_coef(c, yy));
            CK(O::multiaxpy(c, vec(k.Z, 0, y), jy, c->d_coef, x + (long)y * n, (long)nb * n));
            ST(c->sync());
            rel[y] = std::abs(gv[y][jy]) / bnorm[y];
            // reset this system's Hessenberg for the next cycle
            std::fill(H[y].begin(), H[y].end(), cd(0));
        }
        xz = false;
        if (!verify) {
            bool any_left = false;
            for (int y = 0; y < nb; y++)
                if (active[y]) {
                    if (rel[y] <= tol) {
                        active[y] = 0;
                        conv[y] = 1;
                    } else {
                        any_left = true;
                    }
                }
            if (!any_left || its >= maxit) break;
        }
    }
    *iters = its;
    for (int y = 0; y < nb; y++) {
        rel_out[y] = conv[y] ? std::min(rel[y], tol) : rel[y];
        conv_out[y] = conv[y];
    }
    return OVL_OK;
}

// SAP-preconditioned batched Wilson solve (precision T), tolerance eps for every system.
template <typename T>
ovl_status wilson_solve_batch(Ctx *c, int nb, const T *in, T *out, double m0, double eps, const char *active) {
    Krylov<T> &k = sizeof(T) == 8 ? (Krylov<T> &)c->kbo_wil64 : (Krylov<T> &)c->kbo_wil32;
    int &cap = c->kb_n[sizeof(T) == 8 ? 3 : 2];
    ST(ensure_krylov_batch<T>(c, k, cap, std::min(c->p.prec_restart, 16), nb));
    T *&scratch = sizeof(T) == 8 ? (T *&)c->sap_r64 : (T *&)c->sap_r32;
    if (!scratch) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(T)));
        scratch = (T *)buf;
    }
    SapGeom sg = make_sap_geom(c->g, c->p.sap_block);
    sg.tps = c->sap_tps;
    const long n = c->n64;
    auto mv = [&](const T *a, T *o, const double *) -> ovl_status {
        if (sizeof(T) == 8)
            CK(wilson_batch_f64(c->g, c->U64, (const double2 *)a, (double2 *)o, (long)c->g.V * 12, nb, m0, 0, 1.0,
                                nullptr, 0.0, c->stream));
        else
            CK(wilson_batch_f32(c->g, c->U32, (const float4 *)a, (float4 *)o, (long)c->g.V * 6, nb, (float)m0, 0,
                                1.f, nullptr, 0.f, c->stream));
        return OVL_OK;
    };
    auto pc = [&](const T *a, T *o, const char *act) -> ovl_status {
        for (int y = 0; y < nb; y++) {
            if (!act[y]) CK(cudaMemsetAsync(o + (long)y * n, 0, n * sizeof(T), c->stream));
            else if (sizeof(T) == 4 && c->p.wilson_mg)
                ST(mg_apply_f32(c, (const float4 *)(a + (long)y * n), (float4 *)(o + (long)y * n), m0));
            else CK(Ops<T>::sap(c, sg, a + (long)y * n, o + (long)y * n, scratch, m0));
        }
        return OVL_OK;
    };
    int its;
    std::vector<double> rel(nb);
    std::unique_ptr<bool[]> conv(new bool[nb]);
    (void)active;
    ST(fgmres_batch<T>(c, k, nb, out, in, eps, c->p.prec_max_iter, true, mv, pc, &its, rel.data(), conv.get(),
                       false));
    c->stat_prec += (long)its * nb;
    return OVL_OK;
}

}  // namespace

// Bytes of device memory one batched right-hand side needs (Krylov bases, multishift and
// staging vectors) with the restart lengths the batched solver uses.
static size_t batch_bytes_per_rhs(const Ctx *c) {
    const double v64 = (double)c->n64 * 8.0, v32 = (double)c->n64 * 4.0;
    const int mo = std::min(c->p.restart, 32), mi = std::min(c->p.restart_inner, 32), mw = std::min(c->p.prec_restart, 16);
    double b = (2 * mo + 3) * v64 + (c->npole + 3) * v64 + 2 * v64;                 // outer + FP64 multishift + x, b
    b += (2 * mi + 3) * v32 + (2 * mw + 3) * v32 + (c->npole + 3) * v32 + 2 * v32;  // inner, Wilson, FP32 multishift
    return (size_t)b;
}

int batch_size_for(Ctx *c, int want) {
    if (c->fixed_batch) return std::max(1, std::min(want, kMaxBatch));
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    const size_t per = batch_bytes_per_rhs(c);
    // keep 10% of the device (at least 8 GB) free for staging and later calls
    const size_t keep = std::max((size_t)8 << 30, tot / 10);
    const size_t budget = fr > keep ? fr - keep : 0;
    int nb = std::min(want, kMaxBatch);
    while (nb > 1 && per * (size_t)nb > budget) nb--;
    return nb;
}

ovl_status solve_batch(Ctx *c, double2 *x, const double2 *b, int nb, double tol, int *outer_iters, double *worst_res,
                       bool *all_conv) {
    const long n = c->n64;
    ST(ensure_krylov_batch<double>(c, c->kbo_outer, c->kb_n[0], std::min(c->p.restart, 32), nb));
    const bool mixed = c->p.precision != OVL_FP64 || c->p.precond == OVL_PREC_RECURSIVE;
    // FP32 staging for nb vectors
    float *fa = nullptr, *fb = nullptr;
    {
        static_assert(sizeof(float4) == 16, "");
        if (!c->fbat || c->fbat_cap < nb) {
            void *buf;
            ST(c->alloc(&buf, (size_t)n * sizeof(float) * 2 * nb));
            c->fbat = (float *)buf;
            c->fbat_cap = nb;
        }
        fa = c->fbat;
        fb = c->fbat + (long)nb * n;
    }
    const double tight = std::max(1e-14, std::min(c->p.sign_tol, 0.1 * tol));
    const double low_ok = low_sign_floor(c->p.precision);
    // inner batched FP32 FGMRES on D_N, preconditioned by the batched Wilson solve
    auto inner = [&](const float *in, float *out, const char *act) -> ovl_status {
        ST(ensure_krylov_batch<float>(c, c->kbo_inner, c->kb_n[1], std::min(c->p.restart_inner, 32), nb));
        const double eps = c->p.eps_inner;
        auto mv = [&](const float *a, float *o, const double *relv) -> ovl_status {
            double t[kMaxBatch];
            for (int y = 0; y < nb; y++)
                t[y] = relv[y] >= 1.5 ? 0.0 : relax_tol(c, eps, relv[y] < 0 ? eps : relv[y], 1e-6, 1e-1);
            return c->sign32_batch((const float4 *)a, (float4 *)o, nb, t, 1);
        };
        auto pc = [&](const float *a, float *o, const char *act2) -> ovl_status {
            CK(zero_inactive<float>(c, const_cast<float *>(a), nb, act2));
            return wilson_solve_batch<float>(c, nb, a, o, c->m0_prec, c->p.eps_prec, act2);
        };
        int its;
        std::vector<double> rel(nb);
        std::unique_ptr<bool[]> conv(new bool[nb]);
        (void)act;
        ST(fgmres_batch<float>(c, c->kbo_inner, nb, out, in, eps, c->p.max_inner, true, mv, pc, &its, rel.data(),
                               conv.get(), false));
        c->stat_inner += its * nb;
        return OVL_OK;
    };
    auto mv = [&](const double *a, double *o, const double *relv) -> ovl_status {
        double t[kMaxBatch];
        bool low = mixed;
        for (int y = 0; y < nb; y++) {
            if (relv[y] >= 1.5) t[y] = 0.0;   // converged system: no work
            else t[y] = relv[y] < 0 ? tight : relax_tol(c, tol, relv[y], tight, 1e-1);
            if (t[y] > 0 && (relv[y] < 0 || t[y] < low_ok)) low = false;
        }
        if (low) {
            CK(spinor_d2f_n(c, (const double2 *)a, (float4 *)fa, nb));
            ST(c->sign32_batch((const float4 *)fa, (float4 *)fb, nb, t, 1));
            CK(spinor_f2d_n(c, (const float4 *)fb, (double2 *)o, nb));
            return OVL_OK;
        }
        return c->sign_outer_batch((const double2 *)a, (double2 *)o, nb, t, 1);
    };
    auto pc = [&](const double *a, double *o, const char *act) -> ovl_status {
        if (!mixed && c->p.precond == OVL_PREC_WILSON) {
            CK(zero_inactive<double>(c, const_cast<double *>(a), nb, act));
            return wilson_solve_batch<double>(c, nb, a, o, c->m0_prec, c->p.eps_prec, act);
        }
        if (c->p.precond == OVL_PREC_NONE) {
            CK(cudaMemcpyAsync(o, a, (size_t)nb * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            return OVL_OK;
        }
        CK(spinor_d2f_n(c, (const double2 *)a, (float4 *)fa, nb));
        CK(zero_inactive<float>(c, fa, nb, act));
        if (c->p.precond == OVL_PREC_WILSON) ST(wilson_solve_batch<float>(c, nb, fa, fb, c->m0_prec, c->p.eps_prec, act));
        else ST(inner(fa, fb, act));
        CK(spinor_f2d_n(c, (const float4 *)fb, (double2 *)o, nb));
        return OVL_OK;
    };
    // x holds the initial guesses; start from zero when all of them are zero
    double nx = 0.0;
    for (int y = 0; y < nb; y++) {
        double v;
        ST(c->norm2_d((const double *)(x + (long)y * (n / 2)), &v));
        nx += v;
    }
    int its;
    std::vector<double> rel(nb);
    std::unique_ptr<bool[]> conv(new bool[nb]);
    ST(fgmres_batch<double>(c, c->kbo_outer, nb, (double *)x, (const double *)b, tol, c->p.max_iter, nx == 0.0, mv,
                            pc, &its, rel.data(), conv.get(), true));
    *outer_iters = its * nb;
    *worst_res = 0.0;
    *all_conv = true;
    for (int y = 0; y < nb; y++) {
        *worst_res = std::max(*worst_res, rel[y]);
        *all_conv = *all_conv && conv[y];
    }
    return OVL_OK;
}

}  // namespace ovl

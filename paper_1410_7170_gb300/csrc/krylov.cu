// Restarted Krylov sign function with thick restarts (Sec. 5.2), FP64.
//
// Sec. 5.2 evaluates sign(Gamma5 D_W) chi with a restarted Krylov method for matrix
// functions that allows thick restarts (quadrature-based restarts, Frommer, Guettel and
// Schweitzer 2014). For Hermitian Q:
//
//   sign(Q) b = f(A) c,   A = Q^2,  c = Q b,  f(z) = z^{-1/2} = (2/pi) int_0^inf ds / (z + s^2).
//
// Quadrature: s = e^u and the trapezoidal rule in u (step 0.2, truncated 37 units beyond
// ln sqrt of the ends of the spectrum of A) give f(z) ~ sum_j w_j / (z + t_j) to rounding
// on the whole interval [lam_min^2, lam_max^2].
//
// Each cycle extends an orthonormal basis W of at most m vectors by Lanczos steps with
// A (two-pass classical Gram-Schmidt against the whole basis, on the device) and forms
// H = W^H A W from the coefficients. The error of the current approximation f is
//   sum_j w_j xi_j (A + t_j)^{-1} W e_s,
// the Galerkin step on W adds W sum_j w_j xi_j (H + t_j)^{-1} e_s to f, and the residual
// of that step is collinear with the next basis vector w_m:
//   xi_j <- -xi_j beta (e_{m-1}^T (H + t_j)^{-1} e_s).
// With ||(A + t)^{-1}|| <= 1/(lam_min^2 + t) the error is at most
//   sum_j w_j |xi_j| / (lam_min^2 + t_j),
// and the iteration stops when that bound is <= tol ||b||. (H + t_j)^{-1} e_s comes from
// one eigendecomposition of H per cycle (on the host), for all nodes at once.
//
// Thick restart: the next basis starts with the Ritz vectors W S e_i of the krylov_keep
// smallest Ritz values theta_i of H, then w_m (s = krylov_keep); A W S e_i =
// theta_i W S e_i + beta S_{m-1,i} w_m makes the new projected matrix diag(theta) bordered
// by beta S_{m-1,i} in row s; Gram-Schmidt fills column s. Without kept vectors the
// method is the plain quadrature-based restart (s = 0).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "internal.h"
#include "solver.h"

namespace ovl {

namespace {

using cdx = std::complex<double>;

// out = gamma5 x + r y on the internal FP64 layout double2 [p][12][Vh] (gamma5 flips the
// sign of spins 0 and 1, components c < 6); y nullable (then out = gamma5 x).
__global__ void k_g5_axpy_f64(const double2 *__restrict__ x, double r, const double2 *__restrict__ y,
                              double2 *__restrict__ out, long Vh) {
    const long n = 24 * Vh;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int c = (int)((k / Vh) % 12);
        double2 v = x[k];
        if (c < 6) {
            v.x = -v.x;
            v.y = -v.y;
        }
        if (y) {
            const double2 u = y[k];
            v.x = fma(r, u.x, v.x);
            v.y = fma(r, u.y, v.y);
        }
        out[k] = v;
    }
}

constexpr double kQuadStep = 0.2;
constexpr double kQuadTail = 37.0;

// nodes t_j and weights w_j of sum_j w_j / (z + t_j) ~ z^{-1/2} for z in [a_lo, a_hi]
void quadrature(double a_lo, double a_hi, std::vector<double> &t, std::vector<double> &w) {
    const double u_lo = 0.5 * log(a_lo) - kQuadTail, u_hi = 0.5 * log(a_hi) + kQuadTail;
    const int n = (int)ceil((u_hi - u_lo) / kQuadStep) + 1;
    t.resize(n);
    w.resize(n);
    for (int j = 0; j < n; j++) {
        const double u = u_lo + kQuadStep * j;
        t[j] = exp(2.0 * u);
        w[j] = (2.0 / M_PI) * kQuadStep * exp(u);
    }
}

}  // namespace

ovl_status Ctx::ensure_ksign() {
    if (ks_W) return OVL_OK;
    const int m = p.krylov_m, keep = p.krylov_keep;
    const long words = (long)g.V * 12;
    void *buf;
    ST(alloc(&buf, (size_t)(m + 1 + keep + 2) * words * sizeof(double2)));
    ks_W = (double2 *)buf;
    ks_Y = ks_W + (size_t)(m + 1) * words;
    ks_f = ks_Y + (size_t)keep * words;
    ks_tmp = ks_f + words;
    ST(alloc(&buf, (size_t)2 * m * std::max(keep, 1) * sizeof(double)));
    ks_S = (double *)buf;
    return OVL_OK;
}

ovl_status Ctx::sign64_krylov(const double2 *b, double2 *out, double tol, int mode) {
    PhaseClock pclk(this, &t_sign64);
    Ctx *c = this;
    ST(ensure_ksign());
    const int m = p.krylov_m, keep = p.krylov_keep;
    const long n = n64, words = (long)g.V * 12;
    auto vec = [&](double2 *base, int j) { return base + (size_t)j * words; };
    std::vector<double> dc;
    const double2 *bm = b;
    if (ndefl) {   // as with the rational approximation: the iteration sees Pi b
        ST(defl_project64(b, defl_tmp64, dc));
        bm = defl_tmp64;
    }
    double bb;
    ST(norm2_d((const double *)bm, &bb));
    const double bnorm = sqrt(bb);
    CK(cudaMemsetAsync(ks_f, 0, words * sizeof(double2), stream));
    long matvecs = 0;
    if (bnorm > 0) {
        CK(wilson_f64(g, U64, bm, ks_W, m0_ker, 1, 1.0, nullptr, 0.0, stream));   // c = Q b
        double cc;
        ST(norm2_d((const double *)ks_W, &cc));
        const double cnorm = sqrt(cc);
        if (!(cnorm > 0) || !isfinite(cnorm)) {
            err = "Krylov sign: Q b is zero or not finite";
            return OVL_EBREAKDOWN;
        }
        CK(dev_axpby(1.0 / cnorm, (const double *)ks_W, 0.0, (double *)ks_W, n, stream));
        const double a_lo = lam_min * lam_min, a_hi = lam_max * lam_max;
        std::vector<double> qt, qw;
        quadrature(a_lo, a_hi, qt, qw);
        const int J = (int)qt.size();
        std::vector<cdx> xi(J, cdx(cnorm, 0.0));
        std::vector<cdx> H((size_t)m * m, cdx(0.0));
        std::vector<double> theta(m);
        std::vector<cdx> S((size_t)m * m), A((size_t)m * m);
        int j0 = 0, s = 0;
        while (true) {
            int me = m;
            double beta = 0.0;
            for (int j = j0; j < m; j++) {
                double2 *w = vec(ks_W, j + 1);
                CK(wilson_f64(g, U64, vec(ks_W, j), ks_tmp, m0_ker, 1, 1.0, nullptr, 0.0, stream));
                CK(wilson_f64(g, U64, ks_tmp, w, m0_ker, 1, 1.0, nullptr, 0.0, stream));
                matvecs++;
                for (int pass = 0; pass < 2; pass++) {   // two-pass classical Gram-Schmidt
                    double hc[2 * 128];
                    CK(dev_multidot((const double *)ks_W, n, j + 1, (const double *)w, n, d_scal, d_md_part, stream));
                    ST(fetch(d_scal, 2 * (j + 1), hc));
                    std::vector<cdx> neg(j + 1);
                    for (int i = 0; i <= j; i++) {
                        const cdx h(hc[2 * i], hc[2 * i + 1]);
                        H[(size_t)i * m + j] += h;
                        neg[i] = -h;
                    }
                    ST(upload_coef(c, neg));
                    CK(dev_multiaxpy((const double *)ks_W, n, j + 1, d_coef, (double *)w, n, stream));
                }
                double ww;
                ST(norm2_d((const double *)w, &ww));
                beta = sqrt(ww);
                if (!isfinite(beta)) {
                    err = "Krylov sign: non-finite Lanczos coefficient";
                    return OVL_EBREAKDOWN;
                }
                double hmax = 0.0;
                for (int i = 0; i <= j; i++)
                    for (int l = 0; l <= j; l++) hmax = std::max(hmax, std::abs(H[(size_t)i * m + l]));
                if (beta <= 1e-14 * hmax) {   // invariant subspace: the Galerkin step is exact
                    beta = 0.0;
                    me = j + 1;
                    break;
                }
                CK(dev_axpby(1.0 / beta, (const double *)w, 0.0, (double *)w, n, stream));
                if (j + 1 < m) H[(size_t)(j + 1) * m + j] = beta;
            }
            // eigendecomposition of the Hermitian part of H (me x me)
            for (int i = 0; i < me; i++)
                for (int l = 0; l < me; l++)
                    A[(size_t)i * me + l] = 0.5 * (H[(size_t)i * m + l] + std::conj(H[(size_t)l * m + i]));
            if (hermitian_eig(me, A.data(), theta.data(), S.data()) != 0) {
                err = "Krylov sign: projected eigenproblem did not converge";
                return OVL_ENOCONV;
            }
            // all nodes at once in the eigenbasis: d = (theta + t_j)^{-1} S^H e_s
            std::vector<cdx> acc(me, cdx(0.0));
            double bound = 0.0;
            for (int q = 0; q < J; q++) {
                const cdx wx = qw[q] * xi[q];
                cdx gam(0.0);
                for (int i = 0; i < me; i++) {
                    const cdx d = std::conj(S[(size_t)s * me + i]) / (theta[i] + qt[q]);
                    acc[i] += wx * d;
                    gam += S[(size_t)(me - 1) * me + i] * d;
                }
                xi[q] = -xi[q] * beta * gam;
                bound += qw[q] * std::abs(xi[q]) / (a_lo + qt[q]);
            }
            std::vector<cdx> coef(me, cdx(0.0));
            for (int r = 0; r < me; r++)
                for (int i = 0; i < me; i++) coef[r] += S[(size_t)r * me + i] * acc[i];
            ST(upload_coef(c, coef));
            CK(dev_multiaxpy((const double *)ks_W, n, me, d_coef, (double *)ks_f, n, stream));
            ks_cycles++;
            if (beta == 0.0 || bound <= tol * bnorm) break;
            if (matvecs >= p.max_ms_iter) {
                ks_matvecs += matvecs;
                stat_ms64 += matvecs;
                err = "Krylov sign reached max_ms_iter products with Q^2";
                return OVL_ENOCONV;
            }
            // thick restart: W_0..kk-1 <- Ritz vectors of the kk smallest Ritz values, W_kk <- w_m
            const int kk = std::min(keep, me - 1);
            if (kk > 0) {
                std::vector<double> h((size_t)2 * kk * me);
                for (int i = 0; i < kk; i++)
                    for (int r = 0; r < me; r++) {
                        h[2 * ((size_t)i * me + r)] = S[(size_t)r * me + i].real();
                        h[2 * ((size_t)i * me + r) + 1] = S[(size_t)r * me + i].imag();
                    }
                CK(cudaMemcpyAsync(ks_S, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, stream));
                CK(cudaMemsetAsync(ks_Y, 0, (size_t)kk * words * sizeof(double2), stream));
                for (int i = 0; i < kk; i++)
                    CK(dev_multiaxpy((const double *)ks_W, n, me, ks_S + (size_t)2 * me * i, (double *)vec(ks_Y, i), n,
                                     stream));
                ST(sync());   // h is pageable and local
            }
            CK(cudaMemcpyAsync(vec(ks_W, kk), vec(ks_W, me), words * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
            if (kk > 0)
                CK(cudaMemcpyAsync(ks_W, ks_Y, (size_t)kk * words * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
            std::fill(H.begin(), H.end(), cdx(0.0));
            for (int i = 0; i < kk; i++) {
                H[(size_t)i * m + i] = theta[i];
                H[(size_t)kk * m + i] = beta * S[(size_t)(me - 1) * me + i];
            }
            j0 = kk;
            s = kk;
        }
    }
    ks_matvecs += matvecs;
    stat_ms64 += matvecs;
    if (mode == 0) {
        CK(cudaMemcpyAsync(out, ks_f, words * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
    } else {   // D_N b = rho b + gamma5 sign(Q) b
        k_g5_axpy_f64<<<plain_grid(words), kBlock, 0, stream>>>(ks_f, rho, b, out, g.Vh);
        count_launches(1);
        CK(cudaGetLastError());
    }
    if (ndefl) ST(defl_add64(dc, out, mode));
    return OVL_OK;
}

}  // namespace ovl

// Low-mode deflation of the sign function (Sec. 5.2):
//
//   sign(Q) chi = sum_{i<k} sign(lambda_i) (xi_i^H chi) xi_i + sign(Q) Pi chi,
//   Pi = I - Xi Xi^H,  Q = Gamma5 D_W(m0_ker),
//
// with lambda_1..lambda_k the eigenvalues of Q of smallest modulus and xi_i their
// normalised eigenvectors. The first term is exact; the spectrum seen by the rational
// approximation of the second starts at |lambda_{k+1}|, so its interval shrinks and the
// multishift CG converges faster.
//
// Eigenpairs: a thick-restart Krylov-Schur iteration on the Hermitian positive Q^2, FP64,
// with two-pass classical Gram-Schmidt against the whole basis (so the projected matrix is
// formed from the orthogonalisation coefficients and stays Hermitian to rounding):
//   extend the basis to m vectors; Rayleigh-Ritz on the m x m projected matrix (host
//   eigensolver); a Ritz pair (theta, V s) has residual norm |beta_m s_m|; keep the nkeep
//   smallest Ritz vectors plus the last basis vector (the projected matrix becomes
//   diag(theta) bordered by beta_m s_m) and extend again, until k + 1 pairs converge.
// A final Rayleigh-Ritz step with Q itself on the converged vectors gives the signed
// eigenvalues and eigenvectors of Q; the (k+1)-th |eigenvalue| sets the new lower end of
// the Zolotarev interval.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <numeric>
#include <vector>

#include "internal.h"
#include "solver.h"

namespace ovl {

namespace {

using cdx = std::complex<double>;

// y = gamma5 x on the internal FP64 layout double2 [p][12][Vh]: spins 0 and 1 (components
// c < 6) change sign.
__global__ void k_g5_f64(const double2 *__restrict__ x, double2 *__restrict__ y, long Vh) {
    const long n = 24 * Vh;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const int c = (int)((k / Vh) % 12);
        const double2 v = x[k];
        y[k] = c < 6 ? make_double2(-v.x, -v.y) : v;
    }
}

inline int grid_for(long n) {
    long b = (n + kBlock - 1) / kBlock;
    const long cap = (long)device_sm_count() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// coefficient vectors (host, complex) -> device buffer d (contiguous), one copy, then sync so
// the pinned staging area can be reused
static ovl_status upload_block(Ctx *c, const std::vector<cdx> &v, double *d) {
    std::vector<double> h(2 * v.size());
    for (size_t k = 0; k < v.size(); k++) {
        h[2 * k] = v[k].real();
        h[2 * k + 1] = v[k].imag();
    }
    CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    return c->sync();   // h is pageable and local
}

ovl_status Ctx::deflation_setup() {
    Ctx *c = this;
    const auto t0 = std::chrono::steady_clock::now();
    const int k = p.n_deflate;
    const int want = k + 1;                                   // the (k+1)-th sets the interval
    const int mmax = std::min(2 * want + 32, 120);            // basis size (<= 127 for multi-dot)
    const int nkeep = std::min(want + 16, mmax - 16);         // Ritz vectors kept at a restart
    const long n = n64;                                       // reals per vector
    const long words = (long)g.V * 12;                        // double2 per vector
    const double tol_abs = p.deflate_tol * lam_max * lam_max; // Ritz residual target for Q^2
    void *buf;
    ST(alloc(&buf, (size_t)(mmax + 1 + nkeep + 1) * words * sizeof(double2)));
    double2 *V = (double2 *)buf, *W = V + (size_t)(mmax + 1) * words, *tmp = W + (size_t)nkeep * words;
    ST(alloc(&buf, (size_t)2 * mmax * std::max(mmax, 2 * want) * sizeof(double)));
    double *d_S = (double *)buf;
    auto vec = [&](double2 *base, int j) { return base + (size_t)j * words; };
    auto Q2 = [&](const double2 *in, double2 *out) -> ovl_status {
        CK(wilson_f64(g, U64, in, tmp, m0_ker, 1, 1.0, nullptr, 0.0, stream));
        CK(wilson_f64(g, U64, tmp, out, m0_ker, 1, 1.0, nullptr, 0.0, stream));
        defl_matvecs++;
        return OVL_OK;
    };
    // deterministic start vector
    {
        std::vector<double> h(n);
        uint64_t st = 0x243F6A8885A308D3ull;
        for (long i = 0; i < n; i++) {
            st ^= st << 13; st ^= st >> 7; st ^= st << 17;
            h[i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        }
        CK(cudaMemcpyAsync(V, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, stream));
        ST(sync());
        double nn;
        ST(norm2_d((const double *)V, &nn));
        CK(dev_axpby(1.0 / sqrt(nn), (const double *)V, 0.0, (double *)V, n, stream));
    }
    std::vector<cdx> H((size_t)(mmax + 1) * mmax, cdx(0));   // projected matrix (row-major)
    std::vector<double> theta(mmax);
    std::vector<cdx> S((size_t)mmax * mmax);
    int j0 = 0, nconv = 0;
    double beta = 0.0;
    defl_matvecs = 0;
    for (int restart = 0; restart < 200; restart++) {
        for (int j = j0; j < mmax; j++) {
            double2 *w = vec(V, j + 1);
            ST(Q2(vec(V, j), w));
            for (int pass = 0; pass < 2; pass++) {   // two-pass classical Gram-Schmidt
                double hc[2 * 128];
                CK(dev_multidot((const double *)V, n, j + 1, (const double *)w, n, d_scal, d_md_part, stream));
                ST(fetch(d_scal, 2 * (j + 1), hc));
                std::vector<cdx> neg(j + 1);
                for (int i = 0; i <= j; i++) {
                    const cdx h(hc[2 * i], hc[2 * i + 1]);
                    H[(size_t)i * mmax + j] += h;
                    neg[i] = -h;
                }
                ST(upload_block(c, neg, d_coef));
                CK(dev_multiaxpy((const double *)V, n, j + 1, d_coef, (double *)w, n, stream));
            }
            double ww;
            ST(norm2_d((const double *)w, &ww));
            beta = sqrt(ww);
            H[(size_t)(j + 1) * mmax + j] = beta;
            if (!(beta > 0) || !isfinite(beta)) {
                err = "deflation eigensolver: Krylov breakdown";
                return OVL_EBREAKDOWN;
            }
            CK(dev_axpby(1.0 / beta, (const double *)w, 0.0, (double *)w, n, stream));
        }
        // Rayleigh-Ritz on the Hermitian part of the m x m projected matrix
        std::vector<cdx> A((size_t)mmax * mmax);
        for (int i = 0; i < mmax; i++)
            for (int j = 0; j < mmax; j++)
                A[(size_t)i * mmax + j] = 0.5 * (H[(size_t)i * mmax + j] + std::conj(H[(size_t)j * mmax + i]));
        if (hermitian_eig(mmax, A.data(), theta.data(), S.data()) != 0) {
            err = "deflation eigensolver: projected eigenproblem did not converge";
            return OVL_ENOCONV;
        }
        nconv = 0;
        while (nconv < want && std::abs(beta * S[(size_t)(mmax - 1) * mmax + nconv]) <= tol_abs) nconv++;
        const bool done = nconv >= want;
        const int nvec = done ? want : nkeep;
        // Ritz vectors W_i = V S[:, i], i < nvec
        std::vector<cdx> cols((size_t)nvec * mmax);
        for (int i = 0; i < nvec; i++)
            for (int r = 0; r < mmax; r++) cols[(size_t)i * mmax + r] = S[(size_t)r * mmax + i];
        ST(upload_block(c, cols, d_S));
        CK(cudaMemsetAsync(W, 0, (size_t)nvec * words * sizeof(double2), stream));
        for (int i = 0; i < nvec; i++)
            CK(dev_multiaxpy((const double *)V, n, mmax, d_S + (size_t)2 * mmax * i, (double *)vec(W, i), n, stream));
        if (done) break;
        if (restart == 199) {
            err = "deflation eigensolver: eigenpairs did not converge to deflate_tol";
            return OVL_ENOCONV;
        }
        // thick restart: V_0..nkeep-1 <- Ritz vectors, V_nkeep <- V_m; bordered diagonal
        CK(cudaMemcpyAsync(vec(V, nkeep), vec(V, mmax), words * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
        CK(cudaMemcpyAsync(V, W, (size_t)nkeep * words * sizeof(double2), cudaMemcpyDeviceToDevice, stream));
        std::fill(H.begin(), H.end(), cdx(0));
        for (int i = 0; i < nkeep; i++) {
            H[(size_t)i * mmax + i] = theta[i];
            H[(size_t)nkeep * mmax + i] = beta * S[(size_t)(mmax - 1) * mmax + i];
        }
        j0 = nkeep;
    }
    // Rayleigh-Ritz with Q on the converged vectors: G = W^H Q W, sorted by |eigenvalue|
    std::vector<cdx> G((size_t)want * want);
    for (int j = 0; j < want; j++) {
        CK(wilson_f64(g, U64, vec(W, j), tmp, m0_ker, 1, 1.0, nullptr, 0.0, stream));
        double hc[2 * 128];
        CK(dev_multidot((const double *)W, n, want, (const double *)tmp, n, d_scal, d_md_part, stream));
        ST(fetch(d_scal, 2 * want, hc));
        for (int i = 0; i < want; i++) G[(size_t)i * want + j] = cdx(hc[2 * i], hc[2 * i + 1]);
    }
    for (int i = 0; i < want; i++)
        for (int j = i; j < want; j++) {
            const cdx a = 0.5 * (G[(size_t)i * want + j] + std::conj(G[(size_t)j * want + i]));
            G[(size_t)i * want + j] = a;
            G[(size_t)j * want + i] = std::conj(a);
        }
    std::vector<double> lam(want);
    std::vector<cdx> Z((size_t)want * want);
    if (hermitian_eig(want, G.data(), lam.data(), Z.data()) != 0) {
        err = "deflation eigensolver: Rayleigh-Ritz with Q did not converge";
        return OVL_ENOCONV;
    }
    std::vector<int> order(want);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return fabs(lam[a]) < fabs(lam[b]); });
    // eigenvectors of Q: xi_i = W Z[:, order[i]], i < k
    ST(alloc(&buf, (size_t)2 * k * words * sizeof(double2)));
    defl64 = (double2 *)buf;
    defl64g5 = defl64 + (size_t)k * words;
    std::vector<cdx> cols((size_t)k * want);
    for (int i = 0; i < k; i++)
        for (int r = 0; r < want; r++) cols[(size_t)i * want + r] = Z[(size_t)r * want + order[i]];
    ST(upload_block(c, cols, d_S));
    CK(cudaMemsetAsync(defl64, 0, (size_t)k * words * sizeof(double2), stream));
    for (int i = 0; i < k; i++)
        CK(dev_multiaxpy((const double *)W, n, want, d_S + (size_t)2 * want * i, (double *)(defl64 + (size_t)i * words),
                         n, stream));
    defl_lambda.assign(k, 0.0);
    for (int i = 0; i < k; i++) defl_lambda[i] = lam[order[i]];
    defl_next = fabs(lam[order[k]]);
    // gamma5 xi_i (for D_N = rho + gamma5 sign(Q)) and FP32 copies of both
    for (int i = 0; i < k; i++) {
        k_g5_f64<<<grid_for(words * 2), kBlock, 0, stream>>>(defl64 + (size_t)i * words, defl64g5 + (size_t)i * words,
                                                              g.Vh);
        count_launches(1);
    }
    CK(cudaGetLastError());
    ST(alloc(&buf, (size_t)(2 * k + 1) * g.V * 6 * sizeof(float4)));
    defl32 = (float4 *)buf;
    defl32g5 = defl32 + (size_t)k * g.V * 6;
    defl_tmp32 = defl32g5 + (size_t)k * g.V * 6;
    ST(alloc(&buf, (size_t)words * sizeof(double2)));
    defl_tmp64 = (double2 *)buf;
    for (int i = 0; i < 2 * k; i++) CK(spinor_d2f(g, defl64 + (size_t)i * words, defl32 + (size_t)i * g.V * 6, stream));
    // residuals ||Q xi - lambda xi|| of the deflated pairs
    defl_resid = 0.0;
    for (int i = 0; i < k; i++) {
        CK(wilson_f64(g, U64, defl64 + (size_t)i * words, tmp, m0_ker, 1, 1.0, defl64 + (size_t)i * words,
                      -defl_lambda[i], stream));
        double rr;
        ST(norm2_d((const double *)tmp, &rr));
        defl_resid = std::max(defl_resid, sqrt(rr));
    }
    // the Krylov workspace is no longer needed
    for (void *q : {(void *)V, (void *)d_S}) {
        cudaFree(q);
        allocs.erase(std::find(allocs.begin(), allocs.end(), q));
    }
    ndefl = k;
    defl_setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return sync();
}

// bp = Pi b = b - Xi (Xi^H b); coef[2i..2i+1] = xi_i^H b
ovl_status Ctx::defl_project64(const double2 *b, double2 *bp, std::vector<double> &coef) {
    Ctx *c = this;
    const long n = n64;
    coef.assign(2 * ndefl, 0.0);
    CK(dev_multidot((const double *)defl64, n, ndefl, (const double *)b, n, d_scal, d_md_part, stream));
    ST(fetch(d_scal, 2 * ndefl, coef.data()));
    std::vector<cdx> neg(ndefl);
    for (int i = 0; i < ndefl; i++) neg[i] = -cdx(coef[2 * i], coef[2 * i + 1]);
    if (bp != b) CK(cudaMemcpyAsync(bp, b, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    ST(upload_block(c, neg, d_coef));
    CK(dev_multiaxpy((const double *)defl64, n, ndefl, d_coef, (double *)bp, n, stream));
    return OVL_OK;
}

// out += sum_i sign(lambda_i) coef_i xi_i (mode 0: sign(Q) b) or the same with gamma5 xi_i
// (mode 1: the gamma5 sign(Q) b term of D_N b)
ovl_status Ctx::defl_add64(const std::vector<double> &coef, double2 *out, int mode) {
    Ctx *c = this;
    std::vector<cdx> a(ndefl);
    for (int i = 0; i < ndefl; i++) a[i] = (defl_lambda[i] > 0 ? 1.0 : -1.0) * cdx(coef[2 * i], coef[2 * i + 1]);
    ST(upload_block(c, a, d_coef));
    CK(dev_multiaxpy((const double *)(mode == 1 ? defl64g5 : defl64), n64, ndefl, d_coef, (double *)out, n64,
                     stream));
    return OVL_OK;
}

ovl_status Ctx::defl_project32(const float4 *b, float4 *bp, std::vector<double> &coef) {
    Ctx *c = this;
    const long n = n64;
    coef.assign(2 * ndefl, 0.0);
    CK(dev_multidot_f((const float *)defl32, n, ndefl, (const float *)b, n, d_scal, d_md_part, stream));
    ST(fetch(d_scal, 2 * ndefl, coef.data()));
    std::vector<cdx> neg(ndefl);
    for (int i = 0; i < ndefl; i++) neg[i] = -cdx(coef[2 * i], coef[2 * i + 1]);
    if (bp != b) CK(cudaMemcpyAsync(bp, b, n * sizeof(float), cudaMemcpyDeviceToDevice, stream));
    ST(upload_block(c, neg, d_coef));
    CK(dev_multiaxpy_f((const float *)defl32, n, ndefl, d_coef, (float *)bp, n, stream));
    return OVL_OK;
}

ovl_status Ctx::defl_add32(const std::vector<double> &coef, float4 *out, int mode) {
    Ctx *c = this;
    std::vector<cdx> a(ndefl);
    for (int i = 0; i < ndefl; i++) a[i] = (defl_lambda[i] > 0 ? 1.0 : -1.0) * cdx(coef[2 * i], coef[2 * i + 1]);
    ST(upload_block(c, a, d_coef));
    CK(dev_multiaxpy_f((const float *)(mode == 1 ? defl32g5 : defl32), n64, ndefl, d_coef, (float *)out, n64,
                       stream));
    return OVL_OK;
}

}  // namespace ovl

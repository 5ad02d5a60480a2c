// Eigen-decomposition of a small complex Hermitian matrix on the host, for the Rayleigh-Ritz
// steps of the low-mode eigensolver and of the restarted Krylov sign function (orders up to
// ~120, once per restart cycle).
//
// 1. Householder reduction to tridiagonal form (Golub and Van Loan, Matrix Computations,
//    Sec. 8.3.1): for column k the reflector H = I - 2 v v^H maps A[k+1:, k] onto
//    -phi alpha e_1 (alpha its norm, phi the phase of its first entry); the trailing block
//    becomes B - 2 v q^H - 2 q v^H with p = B v, K = v^H p, q = p - K v. The reflectors
//    accumulate into Q (A = Q T Q^H).
// 2. A diagonal unitary D (d_0 = 1, d_{i+1} = d_i s_i/|s_i| for the subdiagonal s_i) makes
//    T real: D^H T D has subdiagonal |s_i|, and Q D carries the phases.
// 3. Implicit symmetric QR steps with the Wilkinson shift (ibid., Sec. 8.3.3) on the
//    unreduced blocks of the real tridiagonal matrix, chasing the bulge with Givens
//    rotations that are applied to the columns of Q D. A subdiagonal entry is set to zero
//    once it is below 2^-52 (|d_i| + |d_{i+1}|).
// Eigenvalues are returned in ascending order with their eigenvectors.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <complex>
#include <numeric>
#include <vector>

namespace ovl {

using cdh = std::complex<double>;

// A: n x n Hermitian, row-major (overwritten). w: eigenvalues ascending; Z: n x n row-major,
// column j the eigenvector of w[j]. Returns 0 on convergence, 1 otherwise.
int hermitian_eig(int n, cdh *A, double *w, cdh *Z) {
    auto a = [&](int i, int j) -> cdh & { return A[(size_t)i * n + j]; };
    std::vector<cdh> Q((size_t)n * n, cdh(0)), v(n), p(n);
    auto q = [&](int i, int j) -> cdh & { return Q[(size_t)i * n + j]; };
    for (int i = 0; i < n; i++) q(i, i) = 1.0;
    // 1. Householder tridiagonalisation
    for (int k = 0; k + 2 < n; k++) {
        const int r = n - k - 1;   // trailing block A[k+1:, k+1:]
        double alpha2 = 0.0;
        for (int i = 0; i < r; i++) alpha2 += std::norm(a(k + 1 + i, k));
        const double alpha = sqrt(alpha2);
        if (alpha == 0.0) continue;
        const cdh x0 = a(k + 1, k);
        const double ax0 = std::abs(x0);
        const cdh phi = ax0 > 0.0 ? x0 / ax0 : cdh(1.0);
        const double vnorm = sqrt(2.0 * alpha * (alpha + ax0));
        for (int i = 0; i < r; i++) v[i] = a(k + 1 + i, k) / vnorm;
        v[0] += phi * alpha / vnorm;
        cdh K(0.0);
        for (int i = 0; i < r; i++) {
            cdh s(0.0);
            for (int j = 0; j < r; j++) s += a(k + 1 + i, k + 1 + j) * v[j];
            p[i] = s;
            K += std::conj(v[i]) * s;
        }
        const double Kr = K.real();
        for (int i = 0; i < r; i++) p[i] -= Kr * v[i];   // q = p - K v
        for (int i = 0; i < r; i++)
            for (int j = 0; j < r; j++)
                a(k + 1 + i, k + 1 + j) -= 2.0 * (v[i] * std::conj(p[j]) + p[i] * std::conj(v[j]));
        a(k + 1, k) = -phi * alpha;
        a(k, k + 1) = std::conj(a(k + 1, k));
        for (int i = 1; i < r; i++) a(k + 1 + i, k) = a(k, k + 1 + i) = 0.0;
        for (int i = 0; i < n; i++) {   // Q <- Q H on columns k+1..n-1
            cdh y(0.0);
            for (int j = 0; j < r; j++) y += q(i, k + 1 + j) * v[j];
            for (int j = 0; j < r; j++) q(i, k + 1 + j) -= 2.0 * y * std::conj(v[j]);
        }
    }
    // 2. real tridiagonal form: diagonal d, subdiagonal e (e[i] couples i and i+1)
    std::vector<double> d(n), e(std::max(n - 1, 1), 0.0);
    cdh delta(1.0);
    for (int i = 0; i < n; i++) {
        d[i] = a(i, i).real();
        if (i) for (int r = 0; r < n; r++) q(r, i) *= delta;
        if (i + 1 < n) {
            const cdh s = a(i + 1, i);
            const double as = std::abs(s);
            e[i] = as;
            if (as > 0.0) delta *= s / as;
        }
    }
    // 3. implicit symmetric QR with Wilkinson shifts
    int converged = 1;
    long steps = 0;
    const long max_steps = 60L * n + 100;
    int hi = n - 1;
    while (hi > 0) {
        // deflate negligible subdiagonal entries, find the unreduced block [lo, hi]
        for (int i = 0; i < hi; i++)
            if (fabs(e[i]) <= DBL_EPSILON * (fabs(d[i]) + fabs(d[i + 1])) || fabs(e[i]) < DBL_MIN) e[i] = 0.0;
        while (hi > 0 && e[hi - 1] == 0.0) hi--;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) lo--;
        if (++steps > max_steps) {
            converged = 0;
            break;
        }
        const double dd = 0.5 * (d[hi - 1] - d[hi]), b = e[hi - 1];
        const double mu = d[hi] - b * b / (dd + (dd >= 0.0 ? 1.0 : -1.0) * hypot(dd, b));
        double x = d[lo] - mu, z = e[lo], bulge = 0.0;
        for (int k = lo; k < hi; k++) {
            if (k > lo) {
                x = e[k - 1];
                z = bulge;
            }
            const double rr = hypot(x, z);
            const double c = rr > 0.0 ? x / rr : 1.0, s = rr > 0.0 ? -z / rr : 0.0;
            if (k > lo) e[k - 1] = rr;
            const double ak = d[k], bk = d[k + 1], tk = e[k];
            d[k] = c * c * ak - 2.0 * c * s * tk + s * s * bk;
            d[k + 1] = s * s * ak + 2.0 * c * s * tk + c * c * bk;
            e[k] = c * s * (ak - bk) + (c * c - s * s) * tk;
            if (k + 1 < hi) {
                bulge = -s * e[k + 1];
                e[k + 1] *= c;
            }
            for (int r = 0; r < n; r++) {   // Q D <- Q D G on columns k, k+1
                const cdh zk = q(r, k), zk1 = q(r, k + 1);
                q(r, k) = c * zk - s * zk1;
                q(r, k + 1) = s * zk + c * zk1;
            }
        }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
    for (int j = 0; j < n; j++) {
        w[j] = d[idx[j]];
        for (int i = 0; i < n; i++) Z[(size_t)i * n + j] = q(i, idx[j]);
    }
    return converged ? 0 : 1;
}

}  // namespace ovl

// Eigen-decomposition of a small complex Hermitian matrix on the host (cyclic Jacobi).
//
// Each step annihilates one off-diagonal pair (p, q). With a_pq = |a_pq| e^{i phi},
// tau = (a_qq - a_pp) / (2 |a_pq|) and t = sgn(tau) / (|tau| + sqrt(1 + tau^2)) (the
// smaller root of t^2 + 2 tau t - 1 = 0), c = 1 / sqrt(1 + t^2), s = t c, the unitary
//   R = [[c, s e^{i phi}], [-s e^{-i phi}, c]]   (acting on coordinates p, q)
// makes (R^H A R)_pq = e^{i phi} (|a_pq| (c^2 - s^2) + c s (a_pp - a_qq)) = 0. Sweeps over
// all pairs repeat until the off-diagonal part is below 1e-15 of the matrix norm; the
// accumulated product of the R is the matrix of eigenvectors. Used for the Rayleigh-Ritz
// steps of the low-mode eigensolver (matrices of order <= a few hundred).
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
    std::vector<cdh> V((size_t)n * n, cdh(0));
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    auto at = [&](int i, int j) -> cdh & { return A[(size_t)i * n + j]; };
    double fro = 0.0;
    for (long k = 0; k < (long)n * n; k++) fro += std::norm(A[k]);
    fro = sqrt(fro);
    int converged = 0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) off += std::norm(at(i, j));
        if (sqrt(2.0 * off) <= 1e-15 * fro || fro == 0.0) {
            converged = 1;
            break;
        }
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                const double b = std::abs(at(p, q));
                if (b == 0.0) continue;
                const cdh ph = at(p, q) / b;   // e^{i phi}
                const double tau = (at(q, q).real() - at(p, p).real()) / (2.0 * b);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                const cdh rpq = s * ph, rqp = -s * std::conj(ph);   // R_pq, R_qp; R_pp = R_qq = c
                // A <- A R (columns p, q)
                for (int i = 0; i < n; i++) {
                    const cdh ap = at(i, p), aq = at(i, q);
                    at(i, p) = ap * c + aq * rqp;
                    at(i, q) = ap * rpq + aq * c;
                }
                // A <- R^H A (rows p, q)
                for (int j = 0; j < n; j++) {
                    const cdh ap = at(p, j), aq = at(q, j);
                    at(p, j) = c * ap + std::conj(rqp) * aq;
                    at(q, j) = std::conj(rpq) * ap + c * aq;
                }
                at(p, q) = 0.0;
                at(q, p) = 0.0;
                at(p, p) = at(p, p).real();
                at(q, q) = at(q, q).real();
                for (int i = 0; i < n; i++) {
                    const cdh vp = V[(size_t)i * n + p], vq = V[(size_t)i * n + q];
                    V[(size_t)i * n + p] = vp * c + vq * rqp;
                    V[(size_t)i * n + q] = vp * rpq + vq * c;
                }
            }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return at(a, a).real() < at(b, b).real(); });
    for (int j = 0; j < n; j++) {
        w[j] = at(idx[j], idx[j]).real();
        for (int i = 0; i < n; i++) Z[(size_t)i * n + j] = V[(size_t)i * n + idx[j]];
    }
    return converged ? 0 : 1;
}

}  // namespace ovl

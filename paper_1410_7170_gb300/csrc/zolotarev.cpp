// Zolotarev's best uniform rational approximation of sign(x), computed on the host
// in FP64 with elliptic functions evaluated from the arithmetic-geometric mean.
//
// On [-1/k, -1] u [1, 1/k] the best approximation of type (2n+1, 2n) is
//   R(x) = d0 x prod_{l=1..n} (x^2 + c_{2l}) / (x^2 + c_{2l-1}),
//   c_j  = sn^2(u_j; k') / cn^2(u_j; k'),  u_j = j K(k') / (2n+1),  k' = sqrt(1-k^2).
// Its error 1 - R equioscillates with extrema at both ends of [1, 1/k] of opposite
// sign, so d0 = 2 / (P(1) + P(1/k)) with P(x) = x prod(...), and the uniform error is
// delta = |1 - d0 P(1)|. Partial fractions: R(x) = d0 x (1 + sum_l a_l / (x^2 + c_{2l-1})).
//
// Elliptic functions (Abramowitz & Stegun 17.6 and 16.4): with parameter m = k'^2,
//   K(m) = pi / (2 AGM(1, sqrt(1-m))),
//   sn, cn via the descending AGM sequence a_i, b_i, c_i: phi_N = 2^N a_N u, then
//   phi_{i-1} = (phi_i + asin(c_i sin(phi_i) / a_i)) / 2, sn = sin phi_0, cn = cos phi_0.
#include <math.h>

#include <vector>

namespace ovl {

namespace {

double agm(double a, double b) {
    for (int it = 0; it < 64 && fabs(a - b) > 1e-16 * a; it++) {
        const double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return 0.5 * (a + b);
}

// Complete elliptic integral of the first kind, parameter m in [0, 1).
double ellip_K(double m) { return M_PI / (2.0 * agm(1.0, sqrt(1.0 - m))); }

// sn(u|m), cn(u|m) by the descending AGM (A&S 16.4.3)
void ellip_sncn(double u, double m, double *sn, double *cn) {
    double a[64], c[64];
    a[0] = 1.0;
    double b = sqrt(1.0 - m);
    c[0] = sqrt(m);
    int N = 0;
    while (fabs(c[N]) > 1e-17 && N < 62) {
        const double an = 0.5 * (a[N] + b);
        const double cn_ = 0.5 * (a[N] - b);
        b = sqrt(a[N] * b);
        N++;
        a[N] = an;
        c[N] = cn_;
    }
    double phi = ldexp(a[N] * u, N);
    for (int i = N; i > 0; i--) phi = 0.5 * (phi + asin(c[i] * sin(phi) / a[i]));
    *sn = sin(phi);
    *cn = cos(phi);
}

}  // namespace

// Returns 0 on success, -1 on bad arguments. a, c have room for n entries.
int zolotarev_host(double k, int n, double *d0, double *a, double *c, double *delta) {
    if (!(k > 0.0 && k < 1.0) || n < 1 || n > 64) return -1;
    const double m = 1.0 - k * k;
    const double Kp = ellip_K(m);
    std::vector<double> cc(2 * n + 1);
    for (int j = 1; j <= 2 * n; j++) {
        double sn, cn;
        ellip_sncn(j * Kp / (2 * n + 1), m, &sn, &cn);
        cc[j] = (sn * sn) / (cn * cn);
    }
    auto P = [&](double x) {
        const double t = x * x;
        double r = x;
        for (int l = 1; l <= n; l++) r *= (t + cc[2 * l]) / (t + cc[2 * l - 1]);
        return r;
    };
    const double p1 = P(1.0), pk = P(1.0 / k);
    *d0 = 2.0 / (p1 + pk);
    *delta = fabs(1.0 - *d0 * p1);
    for (int l = 1; l <= n; l++) {
        const double cl = cc[2 * l - 1];
        double num = 1.0, den = 1.0;
        for (int i = 1; i <= n; i++) {
            num *= cc[2 * i] - cl;
            if (i != l) den *= cc[2 * i - 1] - cl;
        }
        a[l - 1] = num / den;
        c[l - 1] = cl;
    }
    return 0;
}

}  // namespace ovl

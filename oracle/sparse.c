/* Sparse FP64 CPU oracle — TEST INFRASTRUCTURE ONLY (tests, smoke check and
 * the benchmark's CPU-baseline leg). Shares nothing with the GPU library.
 *
 * Layouts: lexicographic site s = ((x0*L1 + x1)*L2 + x2)*L3 + x3, x0 = time.
 *   spinor [V][4][3] complex double, gauge [V][4][3][3] complex double
 *   (U[s][mu][a][b] = row a, column b of U_mu(x)).
 *
 * o2_wilson        D_W(m0) straight from Eq. (Wilson-Dirac) of Sec. 2 with
 *                  a = 1: the full 4x4 (I -+ gamma_mu) times the full 3x3 link,
 *                  no spin projection, no even-odd split, no link compression.
 * o2_q2_shift      (Q^2 + sigma) psi with Q = Gamma5 D_W (Eq. gamma_5_symmetry)
 * o2_cg_shift      plain conjugate gradients on (Q^2 + sigma) x = b
 * o2_sign_zolo     sign(Q) b by the Zolotarev partial fractions, one plain CG
 *                  per pole (no multishift)
 * o2_overlap       D_N b = rho b + Gamma5 sign(Q) b (Eq. overlap_def)
 *
 * Antiperiodic time boundary: a hop across the x0 boundary is multiplied by -1.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static cplx GM[4][4][4];   /* gamma_mu[row][col], chiral basis, gamma_0 = time */
static double G5D[4];      /* diagonal of gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 */
static int g_ready = 0;

static void init_gamma(void)
{
    if (g_ready) return;
    memset(GM, 0, sizeof GM);
    /* gamma_0 = [[0, I], [I, 0]] */
    GM[0][0][2] = 1; GM[0][1][3] = 1; GM[0][2][0] = 1; GM[0][3][1] = 1;
    /* gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] */
    cplx sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    for (int k = 0; k < 3; k++)
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) {
                GM[k + 1][r][c + 2] = -I * sig[k][r][c];
                GM[k + 1][r + 2][c] = I * sig[k][r][c];
            }
    /* gamma_5 as the product, then keep its diagonal (it is diagonal in this basis) */
    cplx P[4][4], T[4][4];
    memcpy(P, GM[0], sizeof P);
    for (int m = 1; m < 4; m++) {
        for (int r = 0; r < 4; r++)
            for (int c = 0; c < 4; c++) {
                cplx s = 0;
                for (int q = 0; q < 4; q++) s += P[r][q] * GM[m][q][c];
                T[r][c] = s;
            }
        memcpy(P, T, sizeof P);
    }
    for (int r = 0; r < 4; r++) G5D[r] = creal(P[r][r]);
    g_ready = 1;
}

int o2_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void o2_gamma5_diag(double *out4)
{
    init_gamma();
    for (int r = 0; r < 4; r++) out4[r] = G5D[r];
}

static long lex4(const int *x, const int *L)
{
    int y[4];
    for (int i = 0; i < 4; i++) y[i] = ((x[i] % L[i]) + L[i]) % L[i];
    return (((long)y[0] * L[1] + y[1]) * L[2] + y[2]) * L[3] + y[3];
}

void o2_wilson(cplx *out, const cplx *in, const cplx *U, const int *L, double m0, int antiperiodic)
{
    init_gamma();
    const long V = (long)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int x[4];
        long r = s;
        x[3] = r % L[3]; r /= L[3];
        x[2] = r % L[2]; r /= L[2];
        x[1] = r % L[1]; r /= L[1];
        x[0] = (int)r;
        cplx acc[4][3];
        memset(acc, 0, sizeof acc);
        for (int mu = 0; mu < 4; mu++) {
            for (int dir = 0; dir < 2; dir++) {      /* 0: x + mu, 1: x - mu */
                int y[4] = {x[0], x[1], x[2], x[3]};
                y[mu] += dir == 0 ? 1 : -1;
                double ph = 1.0;
                if (antiperiodic && mu == 0) {
                    if (dir == 0 && x[0] == L[0] - 1) ph = -1.0;
                    if (dir == 1 && x[0] == 0) ph = -1.0;
                }
                long sn = lex4(y, L);
                const cplx *psi = in + sn * 12;
                cplx link[3][3];
                if (dir == 0) {
                    const cplx *u = U + (s * 4 + mu) * 9;           /* U_mu(x) */
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) link[a][b] = u[a * 3 + b];
                } else {
                    const cplx *u = U + (sn * 4 + mu) * 9;          /* U_mu(x - mu)^H */
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++) link[a][b] = conj(u[b * 3 + a]);
                }
                const double sg = dir == 0 ? -1.0 : 1.0;          /* I - gamma / I + gamma */
                for (int rs = 0; rs < 4; rs++)
                    for (int cs = 0; cs < 4; cs++) {
                        cplx spin = (rs == cs ? 1.0 : 0.0) + sg * GM[mu][rs][cs];
                        if (spin == 0) continue;
                        for (int a = 0; a < 3; a++) {
                            cplx t = 0;
                            for (int b = 0; b < 3; b++) t += link[a][b] * psi[cs * 3 + b];
                            acc[rs][a] += ph * spin * t;
                        }
                    }
            }
        }
        const cplx *p0 = in + s * 12;
        cplx *o = out + s * 12;
        for (int rs = 0; rs < 4; rs++)
            for (int a = 0; a < 3; a++)
                o[rs * 3 + a] = (m0 + 4.0) * p0[rs * 3 + a] - 0.5 * acc[rs][a];
    }
}

void o2_gamma5(cplx *out, const cplx *in, long V)
{
    init_gamma();
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++)
        for (int rs = 0; rs < 4; rs++)
            for (int a = 0; a < 3; a++) out[s * 12 + rs * 3 + a] = G5D[rs] * in[s * 12 + rs * 3 + a];
}

/* out = (Q^2 + sigma) in, Q = Gamma5 D_W(m0); tmp holds 12V entries */
void o2_q2_shift(cplx *out, const cplx *in, const cplx *U, const int *L, double m0, int ap,
                 double sigma, cplx *tmp)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    o2_wilson(tmp, in, U, L, m0, ap);
    o2_gamma5(tmp, tmp, V);
    o2_wilson(out, tmp, U, L, m0, ap);
    o2_gamma5(out, out, V);
    if (sigma != 0.0) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < 12 * V; i++) out[i] += sigma * in[i];
    }
}

static double norm2(const cplx *a, long n)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long i = 0; i < n; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static double redot(const cplx *a, const cplx *b, long n)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long i = 0; i < n; i++) s += creal(conj(a[i]) * b[i]);
    return s;
}

/* Plain CG on the Hermitian positive (Q^2 + sigma) x = b from x = 0.
 * Stops when ||r|| <= tol ||b||. Returns the iteration count (-1: not converged). */
int o2_cg_shift(cplx *x, const cplx *b, const cplx *U, const int *L, double m0, int ap,
                double sigma, double tol, int maxit)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    const long n = 12 * V;
    cplx *r = malloc(n * sizeof(cplx)), *p = malloc(n * sizeof(cplx));
    cplx *Ap = malloc(n * sizeof(cplx)), *tmp = malloc(n * sizeof(cplx));
    memset(x, 0, n * sizeof(cplx));
    memcpy(r, b, n * sizeof(cplx));
    memcpy(p, b, n * sizeof(cplx));
    double bb = norm2(b, n), rr = bb;
    int it = 0, ok = 0;
    if (bb == 0.0) ok = 1;
    while (!ok && it < maxit) {
        o2_q2_shift(Ap, p, U, L, m0, ap, sigma, tmp);
        double alpha = rr / redot(p, Ap, n);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        double rr_new = norm2(r, n);
        it++;
        if (rr_new <= tol * tol * bb) ok = 1;
        double beta = rr_new / rr;
        rr = rr_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
    }
    free(r); free(p); free(Ap); free(tmp);
    return ok ? it : -1;
}

/* sign(Q) b ~= (d0/lmin) Q [ b + sum_l a_l lmin^2 (Q^2 + lmin^2 c_l)^{-1} b ],
 * one plain CG per pole to relative residual tol. iters[l] receives the CG
 * iteration count of pole l. Returns 0, or -1 if a pole did not converge. */
int o2_sign_zolo(cplx *out, const cplx *b, const cplx *U, const int *L, double m0, int ap,
                 double lmin, double d0, int npole, const double *a, const double *c,
                 double tol, int maxit, int *iters)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    const long n = 12 * V;
    cplx *y = malloc(n * sizeof(cplx)), *xl = malloc(n * sizeof(cplx));
    memcpy(y, b, n * sizeof(cplx));
    int status = 0;
    for (int l = 0; l < npole; l++) {
        int it = o2_cg_shift(xl, b, U, L, m0, ap, lmin * lmin * c[l], tol, maxit);
        if (iters) iters[l] = it;
        if (it < 0) status = -1;
        const double w = a[l] * lmin * lmin;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) y[i] += w * xl[i];
    }
    o2_wilson(out, y, U, L, m0, ap);
    o2_gamma5(out, out, V);
    const double sc = d0 / lmin;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) out[i] *= sc;
    free(y); free(xl);
    return status;
}

/* D_N b = rho b + Gamma5 sign(Q) b */
int o2_overlap(cplx *out, const cplx *b, const cplx *U, const int *L, double m0, int ap,
               double rho, double lmin, double d0, int npole, const double *a,
               const double *c, double tol, int maxit, int *iters)
{
    const long V = (long)L[0] * L[1] * L[2] * L[3];
    int st = o2_sign_zolo(out, b, U, L, m0, ap, lmin, d0, npole, a, c, tol, maxit, iters);
    o2_gamma5(out, out, V);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < 12 * V; i++) out[i] += rho * b[i];
    return st;
}

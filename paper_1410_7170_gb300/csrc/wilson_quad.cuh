// Four threads per site: thread q = t & 3 of a quad computes the hops of direction
// mu = q (forward and backward, Eq. Wilson-Dirac); the four partial hopping sums are
// combined with two xor-shuffles. At small volumes this gives the SMs four times the
// threads of a one-thread-per-site stencil, each with two neighbour gathers instead of
// eight, which hides the gather latency.
//
// The spin projection and reconstruction of wilson_site.cuh, written for a run-time mu
// without divergence: each half spinor component is  s_k + c s_j  with (j, c) picked by
// selects from mu, c in {+1, -1, +i, -i}; the lower two spins of the result are d * a_j.
#pragma once
#include "wilson_site.cuh"

namespace ovl {

// z * c for c = cr + i ci with cr, ci in {-1, 0, 1}
template <typename R>
__device__ __forceinline__ cpx<R> mul_unit(cpx<R> z, R cr, R ci) {
    return cpx<R>{cr * z.re - ci * z.im, cr * z.im + ci * z.re};
}

struct QuadCoef {
    // projection: h0 = s0 + c0 s_{j0}, h1 = s1 + c1 s_{j1}
    int j0, j1;
    float c0r, c0i, c1r, c1i;
    // reconstruction: lower spin 2 += d0 a_{k0}, spin 3 += d1 a_{k1}
    int k0, k1;
    float d0r, d0i, d1r, d1i;
};

// Coefficients for (1 - gamma_mu) (fwd = 1) or (1 + gamma_mu) (fwd = 0) in the chiral basis.
__device__ __forceinline__ QuadCoef quad_coef(int mu, bool fwd) {
    QuadCoef q;
    // projection indices are the same for both signs
    q.j0 = (mu == 0 || mu == 3) ? 2 : 3;
    q.j1 = (mu == 0 || mu == 3) ? 3 : 2;
    const float s = fwd ? 1.f : -1.f;   // (1 + gamma) flips the sign of the gamma part
    // (1 - gamma_mu): mu0: -1,-1  mu1: +i,+i  mu2: +1,-1  mu3: +i,-i
    float a0r = 0, a0i = 0, a1r = 0, a1i = 0;
    if (mu == 0) { a0r = -1; a1r = -1; }
    else if (mu == 1) { a0i = 1; a1i = 1; }
    else if (mu == 2) { a0r = 1; a1r = -1; }
    else { a0i = 1; a1i = -1; }
    q.c0r = s * a0r; q.c0i = s * a0i; q.c1r = s * a1r; q.c1i = s * a1i;
    // reconstruction (1 - gamma): mu0: (0,-1),(1,-1)  mu1: (1,-i),(0,-i)  mu2: (1,-1),(0,+1)  mu3: (0,-i),(1,+i)
    q.k0 = (mu == 0 || mu == 3) ? 0 : 1;
    q.k1 = (mu == 0 || mu == 3) ? 1 : 0;
    float e0r = 0, e0i = 0, e1r = 0, e1i = 0;
    if (mu == 0) { e0r = -1; e1r = -1; }
    else if (mu == 1) { e0i = -1; e1i = -1; }
    else if (mu == 2) { e0r = -1; e1r = 1; }
    else { e0i = -1; e1i = 1; }
    q.d0r = s * e0r; q.d0i = s * e0i; q.d1r = s * e1r; q.d1i = s * e1i;
    return q;
}

template <typename R>
__device__ __forceinline__ void quad_project(const QuadCoef &q, const cpx<R> s[12], cpx<R> h0[3], cpx<R> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<R> sj0 = q.j0 == 2 ? s[6 + c] : s[9 + c];
        const cpx<R> sj1 = q.j1 == 2 ? s[6 + c] : s[9 + c];
        h0[c] = s[c] + mul_unit(sj0, (R)q.c0r, (R)q.c0i);
        h1[c] = s[3 + c] + mul_unit(sj1, (R)q.c1r, (R)q.c1i);
    }
}

template <typename R>
__device__ __forceinline__ void quad_accum(const QuadCoef &q, cpx<R> acc[12], const cpx<R> a0[3], const cpx<R> a1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = acc[c] + a0[c];
        acc[3 + c] = acc[3 + c] + a1[c];
        const cpx<R> ak0 = q.k0 == 0 ? a0[c] : a1[c];
        const cpx<R> ak1 = q.k1 == 0 ? a0[c] : a1[c];
        acc[6 + c] = acc[6 + c] + mul_unit(ak0, (R)q.d0r, (R)q.d0i);
        acc[9 + c] = acc[9 + c] + mul_unit(ak1, (R)q.d1r, (R)q.d1i);
    }
}

// Partial hopping sum of direction mu at site (p, i).
template <typename R, typename LT, typename ST>
__device__ __forceinline__ void wilson_hop_dir(const Geom &g, const LT *__restrict__ U, ST in, int p, int i, int mu,
                                               cpx<R> acc[12]) {
    int x[4];
    eo_coords(g, p, i, x);
    const int q = 1 - p;
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cpx<R>{0, 0};
    const int Lm = g.L[mu], xm = x[mu];
    {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = (xm + 1 == Lm) ? 0 : xm + 1;
        const int j = eo_index(g, y);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        load_link<R>(U, g.Vh, p, mu, i, u);
        const QuadCoef qc = quad_coef(mu, true);
        quad_project(qc, s, h0, h1);
        su3_mul(u, h0, a0);
        su3_mul(u, h1, a1);
        if (mu == 0 && g.antiperiodic && xm == Lm - 1) {
#pragma unroll
            for (int c = 0; c < 3; c++) { a0[c] = -a0[c]; a1[c] = -a1[c]; }
        }
        quad_accum(qc, acc, a0, a1);
    }
    {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = (xm == 0) ? Lm - 1 : xm - 1;
        const int j = eo_index(g, y);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        load_link<R>(U, g.Vh, q, mu, j, u);
        const QuadCoef qc = quad_coef(mu, false);
        quad_project(qc, s, h0, h1);
        su3_dag_mul(u, h0, a0);
        su3_dag_mul(u, h1, a1);
        if (mu == 0 && g.antiperiodic && xm == 0) {
#pragma unroll
            for (int c = 0; c < 3; c++) { a0[c] = -a0[c]; a1[c] = -a1[c]; }
        }
        quad_accum(qc, acc, a0, a1);
    }
}

// Sum acc over the 4 lanes of a quad (all lanes receive the total).
template <typename R>
__device__ __forceinline__ void quad_allreduce(cpx<R> acc[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) {
#pragma unroll
        for (int off = 1; off <= 2; off <<= 1) {
            acc[c].re += __shfl_xor_sync(0xffffffffu, acc[c].re, off);
            acc[c].im += __shfl_xor_sync(0xffffffffu, acc[c].im, off);
        }
    }
}

// Chunk access: a storage word holds CPC complex numbers; a site has 12 / CPC words.
template <typename ST> struct Chunk;
template <> struct Chunk<double2> {
    static constexpr int CPC = 1, NC = 12;
    template <typename R>
    __device__ static void load(const double2 *f, int Vh, int p, int i, int j, cpx<R> v[1]) {
        double2 w = __ldg(f + ((size_t)p * NC + j) * Vh + i);
        v[0] = cpx<R>{(R)w.x, (R)w.y};
    }
    template <typename R>
    __device__ static void store(double2 *f, int Vh, int p, int i, int j, const cpx<R> v[1]) {
        f[((size_t)p * NC + j) * Vh + i] = make_double2((double)v[0].re, (double)v[0].im);
    }
};
template <> struct Chunk<float4> {
    static constexpr int CPC = 2, NC = 6;
    template <typename R>
    __device__ static void load(const float4 *f, int Vh, int p, int i, int j, cpx<R> v[2]) {
        float4 w = __ldg(f + ((size_t)p * NC + j) * Vh + i);
        v[0] = cpx<R>{(R)w.x, (R)w.y};
        v[1] = cpx<R>{(R)w.z, (R)w.w};
    }
    template <typename R>
    __device__ static void store(float4 *f, int Vh, int p, int i, int j, const cpx<R> v[2]) {
        f[((size_t)p * NC + j) * Vh + i] =
            make_float4((float)v[0].re, (float)v[0].im, (float)v[1].re, (float)v[1].im);
    }
};

}  // namespace ovl

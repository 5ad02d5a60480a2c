// One site of the Wilson-Dirac operator, Eq. (Wilson-Dirac) with a = 1:
//
//   (D_W psi)(x) = (m0+4) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                             + (1 + gamma_mu) U_mu(x-mu)^H psi(x-mu) ]
//
// (1 -+ gamma_mu) = 2 pi^-+_mu has rank 2 (Appendix A, Eq. proj_relations): in the
// chiral basis gamma_mu = [[0, A_mu], [A_mu^H, 0]] with A_0 = I, A_k = -i sigma_k,
// (1 - gamma_mu) psi = [h; -A^H h] with h = psi_up - A psi_lo, and
// (1 + gamma_mu) psi = [h; +A^H h] with h = psi_up + A psi_lo.
// So each hop projects to a half spinor h (2 spins x 3 colours), multiplies the two
// colour vectors by the link, and rebuilds the lower two spins with a few sign/i
// swaps: 2 SU(3) x vector products per hop instead of 4.
//
// Antiperiodic time boundary: hops across the x0 boundary carry a factor -1, applied as
// a sign-bit flip of the projected half spinor.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"

namespace ovl {

template <typename R>
__device__ __forceinline__ R fma_r(R a, R b, R c);
template <>
__device__ __forceinline__ double fma_r<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_r<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ ff fma_r<ff>(ff a, ff b, ff c) { return ff_fma(a, b, c); }

// o = u h and o = u^H h as explicit chains of fused multiply-adds: per output real one
// multiply and five FMAs. Summing separately rounded complex products would cost two
// more instructions per output real (the compiler does not reassociate), about a fifth
// of the FP64 stencil's FP64 instructions.
template <typename R>
__device__ __forceinline__ void su3_mul(const cpx<R> u[3][3], const cpx<R> h[3], cpx<R> o[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = u[a][0].re * h[0].re, im = u[a][0].re * h[0].im;
        re = fma_r(-u[a][0].im, h[0].im, re);
        im = fma_r(u[a][0].im, h[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            re = fma_r(u[a][b].re, h[b].re, re);
            im = fma_r(u[a][b].re, h[b].im, im);
            re = fma_r(-u[a][b].im, h[b].im, re);
            im = fma_r(u[a][b].im, h[b].re, im);
        }
        o[a] = cpx<R>{re, im};
    }
}
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const cpx<R> u[3][3], const cpx<R> h[3], cpx<R> o[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        R re = u[0][a].re * h[0].re, im = u[0][a].re * h[0].im;
        re = fma_r(u[0][a].im, h[0].im, re);
        im = fma_r(-u[0][a].im, h[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            re = fma_r(u[b][a].re, h[b].re, re);
            im = fma_r(u[b][a].re, h[b].im, im);
            re = fma_r(u[b][a].im, h[b].im, re);
            im = fma_r(-u[b][a].im, h[b].re, im);
        }
        o[a] = cpx<R>{re, im};
    }
}

// Float-float SU(3) x vector: each output real is a sum of six products, accumulated as one
// running FP32 sum of the leading products (TwoSum keeps it exact) and one FP32 word that
// collects every rounding error and cross term, renormalised once at the end: 12 FP32
// instructions per product against 15 for a renormalised float-float FMA, and a shorter
// instruction stream (the float-float stencil is large enough to miss the instruction cache).
struct ff_dot {
    float s, e;
    __device__ __forceinline__ void first(ff a, ff b) {
        s = __fmul_rn(a.hi, b.hi);
        e = __fmaf_rn(a.hi, b.hi, -s);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
    }
    __device__ __forceinline__ void add(ff a, ff b) {
        const float p = __fmul_rn(a.hi, b.hi);
        const float ep = __fmaf_rn(a.hi, b.hi, -p);
        const ff t = ff_two_sum(s, p);
        s = t.hi;
        e = __fadd_rn(e, __fadd_rn(t.lo, ep));
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
    }
    __device__ __forceinline__ ff done() const { return ff_fast_two_sum(s, e); }
};
template <>
__device__ __forceinline__ void su3_mul<ff>(const cpx<ff> u[3][3], const cpx<ff> h[3], cpx<ff> o[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ff_dot re, im;
        re.first(u[a][0].re, h[0].re);
        im.first(u[a][0].re, h[0].im);
        re.add(-u[a][0].im, h[0].im);
        im.add(u[a][0].im, h[0].re);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            re.add(u[a][b].re, h[b].re);
            im.add(u[a][b].re, h[b].im);
            re.add(-u[a][b].im, h[b].im);
            im.add(u[a][b].im, h[b].re);
        }
        o[a] = cpx<ff>{re.done(), im.done()};
    }
}
template <>
__device__ __forceinline__ void su3_dag_mul<ff>(const cpx<ff> u[3][3], const cpx<ff> h[3], cpx<ff> o[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ff_dot re, im;
        re.first(u[0][a].re, h[0].re);
        im.first(u[0][a].re, h[0].im);
        re.add(u[0][a].im, h[0].im);
        im.add(-u[0][a].im, h[0].re);
#pragma unroll
        for (int b = 1; b < 3; b++) {
            re.add(u[b][a].re, h[b].re);
            im.add(u[b][a].re, h[b].im);
            re.add(u[b][a].im, h[b].im);
            im.add(-u[b][a].im, h[b].re);
        }
        o[a] = cpx<ff>{re.done(), im.done()};
    }
}

// Accumulation of hop contributions: a + b, except in float-float, where the hop
// accumulator is summed without renormalising (TwoSum of the leading words, FP32 sum of the
// rest: 8 instructions instead of 11); wilson_combine renormalises the result.
template <typename R>
__device__ __forceinline__ cpx<R> cadd_acc(cpx<R> a, cpx<R> b) { return a + b; }
__device__ __forceinline__ ff ff_add_lazy(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
template <>
__device__ __forceinline__ cpx<ff> cadd_acc<ff>(cpx<ff> a, cpx<ff> b) {
    return cpx<ff>{ff_add_lazy(a.re, b.re), ff_add_lazy(a.im, b.im)};
}

// -x where neg != 0, by flipping the sign bit (integer pipe, exact)
__device__ __forceinline__ double flip_sign(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}
__device__ __forceinline__ float flip_sign(float x, bool neg) {
    return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000u : 0));
}
__device__ __forceinline__ ff flip_sign(ff x, bool neg) { return ff(flip_sign(x.hi, neg), flip_sign(x.lo, neg)); }
template <typename R>
__device__ __forceinline__ void flip_half(cpx<R> h0[3], cpx<R> h1[3], bool neg) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        h0[c] = cpx<R>{flip_sign(h0[c].re, neg), flip_sign(h0[c].im, neg)};
        h1[c] = cpx<R>{flip_sign(h1[c].re, neg), flip_sign(h1[c].im, neg)};
    }
}

// Forward hop, spin part (1 - gamma_mu): project psi(x+mu) to h0, h1.
template <typename R>
__device__ __forceinline__ void proj_fwd(int mu, const cpx<R> s[12], cpx<R> h0[3], cpx<R> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<R> s0 = s[c], s1 = s[3 + c], s2 = s[6 + c], s3 = s[9 + c];
        switch (mu) {
            case 0: h0[c] = s0 - s2;          h1[c] = s1 - s3;          break;
            case 1: h0[c] = s0 + mul_i(s3);   h1[c] = s1 + mul_i(s2);   break;
            case 2: h0[c] = s0 + s3;          h1[c] = s1 - s2;          break;
            default: h0[c] = s0 + mul_i(s2);  h1[c] = s1 - mul_i(s3);   break;
        }
    }
}
// Forward hop: add [a0; a1; -A^H (a0, a1)] into acc (First: acc is empty, assign).
template <bool First, typename R>
__device__ __forceinline__ void acc_fwd(int mu, cpx<R> acc[12], const cpx<R> a0[3], const cpx<R> a1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        cpx<R> l2, l3;   // lower two spins of the contribution
        switch (mu) {
            case 0: l2 = -a0[c];        l3 = -a1[c];        break;
            case 1: l2 = mul_mi(a1[c]); l3 = mul_mi(a0[c]); break;
            case 2: l2 = -a1[c];        l3 = a0[c];         break;
            default: l2 = mul_mi(a0[c]); l3 = mul_i(a1[c]); break;
        }
        if (First) {
            acc[c] = a0[c];
            acc[3 + c] = a1[c];
            acc[6 + c] = l2;
            acc[9 + c] = l3;
        } else {
            acc[c] = cadd_acc(acc[c], a0[c]);
            acc[3 + c] = cadd_acc(acc[3 + c], a1[c]);
            acc[6 + c] = cadd_acc(acc[6 + c], l2);
            acc[9 + c] = cadd_acc(acc[9 + c], l3);
        }
    }
}
// Backward hop, spin part (1 + gamma_mu).
template <typename R>
__device__ __forceinline__ void proj_bwd(int mu, const cpx<R> s[12], cpx<R> h0[3], cpx<R> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<R> s0 = s[c], s1 = s[3 + c], s2 = s[6 + c], s3 = s[9 + c];
        switch (mu) {
            case 0: h0[c] = s0 + s2;          h1[c] = s1 + s3;          break;
            case 1: h0[c] = s0 + mul_mi(s3);  h1[c] = s1 + mul_mi(s2);  break;
            case 2: h0[c] = s0 - s3;          h1[c] = s1 + s2;          break;
            default: h0[c] = s0 + mul_mi(s2); h1[c] = s1 + mul_i(s3);   break;
        }
    }
}
// Backward hop: add [a0; a1; +A^H (a0, a1)] into acc.
template <typename R>
__device__ __forceinline__ void acc_bwd(int mu, cpx<R> acc[12], const cpx<R> a0[3], const cpx<R> a1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = cadd_acc(acc[c], a0[c]);
        acc[3 + c] = cadd_acc(acc[3 + c], a1[c]);
        switch (mu) {
            case 0: acc[6 + c] = cadd_acc(acc[6 + c], a0[c]);        acc[9 + c] = cadd_acc(acc[9 + c], a1[c]);        break;
            case 1: acc[6 + c] = cadd_acc(acc[6 + c], mul_i(a1[c])); acc[9 + c] = cadd_acc(acc[9 + c], mul_i(a0[c])); break;
            case 2: acc[6 + c] = cadd_acc(acc[6 + c], a1[c]);        acc[9 + c] = cadd_acc(acc[9 + c], -a0[c]);       break;
            default: acc[6 + c] = cadd_acc(acc[6 + c], mul_i(a0[c])); acc[9 + c] = cadd_acc(acc[9 + c], mul_mi(a1[c])); break;
        }
    }
}

// The two hops of direction MU at site (p, i) with coordinates x, added into acc
// (First: acc is empty and the forward hop assigns it).
template <int MU, bool First, typename R, typename LT, typename ST>
__device__ __forceinline__ void hop_dir(const Geom &g, const LT *__restrict__ U, ST in, int p, int i, const int x[4],
                                        cpx<R> acc[12]) {
    const int q = 1 - p;
    {   // forward neighbour x + mu, link U_mu(x) stored at (p, i)
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[MU] = (x[MU] + 1 == g.L[MU]) ? 0 : x[MU] + 1;
        const int j = eo_index(g, y);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        load_link<R>(U, g.Vh, p, MU, i, u);
        proj_fwd(MU, s, h0, h1);
        if (MU == 0) flip_half(h0, h1, g.antiperiodic && x[0] == g.L[0] - 1);
        su3_mul(u, h0, a0);
        su3_mul(u, h1, a1);
        acc_fwd<First>(MU, acc, a0, a1);
    }
    {   // backward neighbour x - mu, link U_mu(x - mu)^H stored at (q, j)
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[MU] = (x[MU] == 0) ? g.L[MU] - 1 : x[MU] - 1;
        const int j = eo_index(g, y);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        load_link<R>(U, g.Vh, q, MU, j, u);
        proj_bwd(MU, s, h0, h1);
        if (MU == 0) flip_half(h0, h1, g.antiperiodic && x[0] == 0);
        su3_dag_mul(u, h0, a0);
        su3_dag_mul(u, h1, a1);
        acc_bwd(MU, acc, a0, a1);
    }
}

// The two hops of direction mu (a run-time value) at site (p, i), added into acc. The
// float-float stencil loops over mu with this body instead of unrolling four copies: its
// fully unrolled form runs to more than 12k instructions per site and stalls on instruction
// fetch (measured at 16^4: 87 us per multishift stencil unrolled, 59 us as a loop). The
// link is loaded after the spin projection, so the neighbour spinor is dead before the link
// is live (53 us; 128 registers, two blocks per SM). Neighbour coordinates are formed with
// selects, not by indexing x with mu (that would put x in local memory).
template <typename R, typename LT, typename ST>
__device__ __forceinline__ void hop_dir_rt(const Geom &g, const LT *__restrict__ U, ST in, int p, int i, const int x[4],
                                           int mu, cpx<R> acc[12]) {
    const int q = 1 - p;
    int yf[4], yb[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const bool on = m == mu;
        yf[m] = on ? (x[m] + 1 == g.L[m] ? 0 : x[m] + 1) : x[m];
        yb[m] = on ? (x[m] == 0 ? g.L[m] - 1 : x[m] - 1) : x[m];
    }
    {   // forward neighbour x + mu, link U_mu(x) stored at (p, i)
        const int j = eo_index(g, yf);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        proj_fwd(mu, s, h0, h1);
        flip_half(h0, h1, mu == 0 && g.antiperiodic && x[0] == g.L[0] - 1);
        load_link<R>(U, g.Vh, p, mu, i, u);
        su3_mul(u, h0, a0);
        su3_mul(u, h1, a1);
        acc_fwd<false>(mu, acc, a0, a1);
    }
    {   // backward neighbour x - mu, link U_mu(x - mu)^H stored at (q, j)
        const int j = eo_index(g, yb);
        cpx<R> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<R>(in, g.Vh, q, j, s);
        proj_bwd(mu, s, h0, h1);
        flip_half(h0, h1, mu == 0 && g.antiperiodic && x[0] == 0);
        load_link<R>(U, g.Vh, q, mu, j, u);
        su3_dag_mul(u, h0, a0);
        su3_dag_mul(u, h1, a1);
        acc_bwd(mu, acc, a0, a1);
    }
}

// The hops of direction MU for two input fields at once: each link is loaded (for FP32:
// and its third row rebuilt) once and applied to both.
template <int MU, bool First, typename R, typename LT, typename ST>
__device__ __forceinline__ void hop_dir2(const Geom &g, const LT *__restrict__ U, ST in0, ST in1, int p, int i,
                                         const int x[4], cpx<R> acc0[12], cpx<R> acc1[12]) {
    const int q = 1 - p;
    {   // forward neighbour x + mu, link U_mu(x) stored at (p, i)
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[MU] = (x[MU] + 1 == g.L[MU]) ? 0 : x[MU] + 1;
        const int j = eo_index(g, y);
        const bool neg = MU == 0 && g.antiperiodic && x[0] == g.L[0] - 1;
        cpx<R> u[3][3];
        load_link<R>(U, g.Vh, p, MU, i, u);
#pragma unroll
        for (int f = 0; f < 2; f++) {
            cpx<R> s[12], h0[3], h1[3], a0[3], a1[3];
            load_spinor<R>(f ? in1 : in0, g.Vh, q, j, s);
            proj_fwd(MU, s, h0, h1);
            if (MU == 0) flip_half(h0, h1, neg);
            su3_mul(u, h0, a0);
            su3_mul(u, h1, a1);
            acc_fwd<First>(MU, f ? acc1 : acc0, a0, a1);
        }
    }
    {   // backward neighbour x - mu, link U_mu(x - mu)^H stored at (q, j)
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[MU] = (x[MU] == 0) ? g.L[MU] - 1 : x[MU] - 1;
        const int j = eo_index(g, y);
        const bool neg = MU == 0 && g.antiperiodic && x[0] == 0;
        cpx<R> u[3][3];
        load_link<R>(U, g.Vh, q, MU, j, u);
#pragma unroll
        for (int f = 0; f < 2; f++) {
            cpx<R> s[12], h0[3], h1[3], a0[3], a1[3];
            load_spinor<R>(f ? in1 : in0, g.Vh, q, j, s);
            proj_bwd(MU, s, h0, h1);
            if (MU == 0) flip_half(h0, h1, neg);
            su3_dag_mul(u, h0, a0);
            su3_dag_mul(u, h1, a1);
            acc_bwd(MU, f ? acc1 : acc0, a0, a1);
        }
    }
}

// Hopping sums of two fields at one site (links loaded once for both).
template <typename R, typename LT, typename ST>
__device__ __forceinline__ void wilson_hop2(const Geom &g, const LT *__restrict__ U, ST in0, ST in1, int p, int i,
                                            cpx<R> acc0[12], cpx<R> acc1[12]) {
    int x[4];
    eo_coords(g, p, i, x);
    hop_dir2<0, true, R>(g, U, in0, in1, p, i, x, acc0, acc1);
    hop_dir2<1, false, R>(g, U, in0, in1, p, i, x, acc0, acc1);
    hop_dir2<2, false, R>(g, U, in0, in1, p, i, x, acc0, acc1);
    hop_dir2<3, false, R>(g, U, in0, in1, p, i, x, acc0, acc1);
}

// Hopping sum H(x) = sum_mu [(1-g_mu) U_mu(x) in(x+mu) + (1+g_mu) U_mu(x-mu)^H in(x-mu)]
// for the site (p, i), times -1/2 (the stored links are -1/2 U); `in` is any spinor storage
// accepted by load_spinor.
template <typename R, typename LT, typename ST>
__device__ __forceinline__ void wilson_hop(const Geom &g, const LT *__restrict__ U, ST in, int p, int i,
                                           cpx<R> acc[12]) {
    int x[4];
    eo_coords(g, p, i, x);
    if constexpr (std::is_same<R, ff>::value) {
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = cpx<R>{R(0), R(0)};
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) hop_dir_rt<R>(g, U, in, p, i, x, mu, acc);
    } else {
        hop_dir<0, true, R>(g, U, in, p, i, x, acc);
        hop_dir<1, false, R>(g, U, in, p, i, x, acc);
        hop_dir<2, false, R>(g, U, in, p, i, x, acc);
        hop_dir<3, false, R>(g, U, in, p, i, x, acc);
    }
}

// res = (m0+4) own + hop, where hop (formed with the stored links -1/2 U) is -1/2 times the
// hopping sum H(x): one FMA per real
template <typename R>
__device__ __forceinline__ void wilson_combine(R m4, const cpx<R> own[12], const cpx<R> hop[12], cpx<R> res[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) res[c] = cpx<R>{fma_r(m4, own[c].re, hop[c].re), fma_r(m4, own[c].im, hop[c].im)};
}

}  // namespace ovl

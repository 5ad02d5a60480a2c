// Device-side building blocks: complex arithmetic, even-odd lattice geometry,
// field storage formats and their loads/stores.
//
// Internal layouts (all even-odd, site-major structure-of-arrays so that a warp's
// 32 consecutive sites read 32 consecutive 16-byte words):
//   parity p = (x0+x1+x2+x3) & 1, checkerboard index i = s >> 1 where
//   s = ((x0*L1+x1)*L2+x2)*L3+x3 (needs L3 even); Vh = V/2 sites per parity.
//   FP64 spinor: double2 [p][12 spin-colour][Vh]         (192 B per site)
//   FP32 spinor: float4  [p][6 pairs of spin-colour][Vh] ( 96 B per site)
//   FP16 spinor: uint4 (8 halves) [p][3][Vh] + float norm [p][Vh] (48+4 B per site)
//   BF16 spinor: uint4 (8 bfloat16) [p][3][Vh], no norm              (48 B per site)
//   FP64 link:   double2 [p][mu][9][Vh]   all 18 reals of -1/2 U_mu(x)
//   FP32 link:   float4  [p][mu][3][Vh]   rows 0 and 1 (12 reals) of -1/2 U_mu(x)
// The FP32 stencils rebuild row 2 of an SU(3) link in registers as conj(row0 x row1);
// the FP64 stencils, bound by the FP64 pipes rather than by memory, load all 18 reals
// instead (the rebuild would cost about a fifth of their FP64 instructions).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ovl {

template <typename R>
struct cpx {
    R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// i*a and -i*a
template <typename R>
__device__ __forceinline__ cpx<R> mul_i(cpx<R> a) { return {-a.im, a.re}; }
template <typename R>
__device__ __forceinline__ cpx<R> mul_mi(cpx<R> a) { return {a.im, -a.re}; }
// conj(a)*b
template <typename R>
__device__ __forceinline__ cpx<R> cmul_conj(cpx<R> a, cpx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }

// Lattice geometry shared by all kernels.
struct Geom {
    int L[4];
    int Lh3;    // L3 / 2
    int Vh;     // V / 2
    int V;
    int antiperiodic;
    int tps64, tps32;   // threads per site of the FP64 / FP32 stencils (1 or 4), chosen by the autotuner
    int mrhs32;         // FP32 multi-RHS stencil kernel for <= 6 right-hand sides (1 RHS pairs, 2 tiles of 32
                        // sites, 3 staged links); mrhs32l for 7..12
    int mrhs32l;
    int nsm;            // streaming multiprocessors of the device (grid sizing)
};

// Site visited by thread t of a full-lattice kernel: parities interleave (t even: even
// site, t odd: odd site, same checkerboard index), so the two sites that read a link
// (x and x + mu) and the neighbours of a site are touched close together in time and
// their data is still in L2.
__device__ __forceinline__ void site_of_thread(int t, int &p, int &i) {
    p = t & 1;
    i = t >> 1;
}

// Coordinates of checkerboard site (p, i).
__device__ __forceinline__ void eo_coords(const Geom &g, int p, int i, int x[4]) {
    int x3h = i % g.Lh3;
    int r = i / g.Lh3;
    x[2] = r % g.L[2];
    r /= g.L[2];
    x[1] = r % g.L[1];
    x[0] = r / g.L[1];
    int b = (p + x[0] + x[1] + x[2]) & 1;
    x[3] = 2 * x3h + b;
}

__device__ __forceinline__ int eo_index(const Geom &g, const int x[4]) {
    return (((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3]) >> 1;
}

// ---------------------------------------------------------------------------
// Field storage formats. Each provides load/store of one site's 12 spin-colour
// components as cpx<R>, R the arithmetic type.
// ---------------------------------------------------------------------------
struct SpinorF64 {
    using store_t = double2;
    static constexpr int chunks = 12;
};
struct SpinorF32 {
    using store_t = float4;
    static constexpr int chunks = 6;
};

template <typename R>
__device__ __forceinline__ void load_spinor(const double2 *__restrict__ f, int Vh, int p, int i, cpx<R> s[12]) {
    const double2 *b = f + (size_t)p * 12 * Vh + i;
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 v = __ldg(b + (size_t)c * Vh);
        s[c] = cpx<R>{(R)v.x, (R)v.y};
    }
}
template <typename R>
__device__ __forceinline__ void load_spinor(const float4 *__restrict__ f, int Vh, int p, int i, cpx<R> s[12]) {
    const float4 *b = f + (size_t)p * 6 * Vh + i;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        float4 v = __ldg(b + (size_t)c * Vh);
        s[2 * c] = cpx<R>{(R)v.x, (R)v.y};
        s[2 * c + 1] = cpx<R>{(R)v.z, (R)v.w};
    }
}
template <typename R>
__device__ __forceinline__ void store_spinor(double2 *__restrict__ f, int Vh, int p, int i, const cpx<R> s[12]) {
    double2 *b = f + (size_t)p * 12 * Vh + i;
#pragma unroll
    for (int c = 0; c < 12; c++) b[(size_t)c * Vh] = make_double2((double)s[c].re, (double)s[c].im);
}
template <typename R>
__device__ __forceinline__ void store_spinor(float4 *__restrict__ f, int Vh, int p, int i, const cpx<R> s[12]) {
    float4 *b = f + (size_t)p * 6 * Vh + i;
#pragma unroll
    for (int c = 0; c < 6; c++)
        b[(size_t)c * Vh] = make_float4((float)s[2 * c].re, (float)s[2 * c].im, (float)s[2 * c + 1].re,
                                        (float)s[2 * c + 1].im);
}

// Half-precision spinor: 24 halves per site in 3 uint4 words, scaled by a per-site
// FP32 norm (the largest |component| of the site).
struct HalfSpinor {
    uint4 *v;
    float *norm;
};
struct HalfSpinorC {
    const uint4 *v;
    const float *norm;
};

template <typename R>
__device__ __forceinline__ void load_spinor(HalfSpinorC f, int Vh, int p, int i, cpx<R> s[12]) {
    const uint4 *b = f.v + (size_t)p * 3 * Vh + i;
    const float nrm = __ldg(f.norm + (size_t)p * Vh + i);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint4 w = __ldg(b + (size_t)c * Vh);
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __half2 h = *reinterpret_cast<const __half2 *>(&u[q]);
            float2 fl = __half22float2(h);
            s[4 * c + q] = cpx<R>{(R)(fl.x * nrm), (R)(fl.y * nrm)};
        }
    }
}
template <typename R>
__device__ __forceinline__ void store_spinor(HalfSpinor f, int Vh, int p, int i, const cpx<R> s[12]) {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 12; c++) m = fmaxf(m, fmaxf(fabsf((float)s[c].re), fabsf((float)s[c].im)));
    const float inv = m > 0.f ? 1.0f / m : 0.f;
    uint4 *b = f.v + (size_t)p * 3 * Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint32_t u[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __half2 h = __floats2half2_rn((float)s[4 * c + q].re * inv, (float)s[4 * c + q].im * inv);
            u[q] = *reinterpret_cast<uint32_t *>(&h);
        }
        b[(size_t)c * Vh] = make_uint4(u[0], u[1], u[2], u[3]);
    }
    f.norm[(size_t)p * Vh + i] = m;
}

// BF16 spinor: 24 bfloat16 per site in 3 uint4 words, no scale (BF16 keeps the FP32
// exponent range; 8 significant bits against FP16's 11).
struct Bf16Spinor {
    uint4 *v;
};
struct Bf16SpinorC {
    const uint4 *v;
};

template <typename R>
__device__ __forceinline__ void load_spinor(Bf16SpinorC f, int Vh, int p, int i, cpx<R> s[12]) {
    const uint4 *b = f.v + (size_t)p * 3 * Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint4 w = __ldg(b + (size_t)c * Vh);
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&u[q]);
            float2 fl = __bfloat1622float2(h);
            s[4 * c + q] = cpx<R>{(R)fl.x, (R)fl.y};
        }
    }
}
template <typename R>
__device__ __forceinline__ void store_spinor(Bf16Spinor f, int Vh, int p, int i, const cpx<R> s[12]) {
    uint4 *b = f.v + (size_t)p * 3 * Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint32_t u[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __nv_bfloat162 h = __floats2bfloat162_rn((float)s[4 * c + q].re, (float)s[4 * c + q].im);
            u[q] = *reinterpret_cast<uint32_t *>(&h);
        }
        b[(size_t)c * Vh] = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// Links are stored as V = kLinkScale U: the factor -1/2 of the hopping term of Eq.
// (Wilson-Dirac) is folded into them, so that a site's result (m0+4) psi + hop is one FMA
// per real. For U in SU(3), row 2 = conj(row0 x row1); for V = s U that becomes
// row2(V) = conj(row0(V) x row1(V)) / s.
constexpr double kLinkScale = -0.5;
template <typename R>
__device__ __forceinline__ void reconstruct_row2(cpx<R> u[3][3]) {
    constexpr R inv = (R)(1.0 / kLinkScale);
    u[2][0] = inv * conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
    u[2][1] = inv * conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
    u[2][2] = inv * conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}
constexpr int kLink64Words = 9;   // double2 words per FP64 link
template <typename R>
__device__ __forceinline__ void load_link(const double2 *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    const double2 *b = g + ((size_t)(p * 4 + mu) * kLink64Words) * Vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) {
        double2 v = __ldg(b + (size_t)c * Vh);
        u[c / 3][c % 3] = cpx<R>{(R)v.x, (R)v.y};
    }
}
template <typename R>
__device__ __forceinline__ void load_link(const float4 *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    const float4 *b = g + ((size_t)(p * 4 + mu) * 3) * Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float4 v = __ldg(b + (size_t)c * Vh);
        u[(2 * c) / 3][(2 * c) % 3] = cpx<R>{(R)v.x, (R)v.y};
        u[(2 * c + 1) / 3][(2 * c + 1) % 3] = cpx<R>{(R)v.z, (R)v.w};
    }
    reconstruct_row2(u);
}

// 16-bit links: rows 0 and 1 of -1/2 U (12 reals) in FP16 (LinkH) or BF16 (LinkB), one
// 8-byte word of four 16-bit reals per element, [p][mu][3][Vh] (24 B per link); row 2 is
// rebuilt in FP32 registers. The entries of -1/2 U are bounded by 1/2, so FP16 needs no scale.
struct __align__(8) LinkH {
    uint32_t a, b;
};
struct __align__(8) LinkB {
    uint32_t a, b;
};
__device__ __forceinline__ float2 unpack16(const LinkH *, uint32_t u) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ float2 unpack16(const LinkB *, uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}
__device__ __forceinline__ uint32_t pack16(const LinkH *, float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack16(const LinkB *, float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
template <typename R, typename L16>
__device__ __forceinline__ void load_link16(const L16 *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    const uint2 *b = reinterpret_cast<const uint2 *>(g) + ((size_t)(p * 4 + mu) * 3) * Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const uint2 v = __ldg(b + (size_t)c * Vh);
        const float2 e0 = unpack16(g, v.x), e1 = unpack16(g, v.y);
        u[(2 * c) / 3][(2 * c) % 3] = cpx<R>{(R)e0.x, (R)e0.y};
        u[(2 * c + 1) / 3][(2 * c + 1) % 3] = cpx<R>{(R)e1.x, (R)e1.y};
    }
    reconstruct_row2(u);
}
template <typename R>
__device__ __forceinline__ void load_link(const LinkH *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    load_link16<R>(g, Vh, p, mu, i, u);
}
template <typename R>
__device__ __forceinline__ void load_link(const LinkB *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    load_link16<R>(g, Vh, p, mu, i, u);
}

// gamma_5 = diag(-1,-1,+1,+1) in the chiral basis: flips spins 0 and 1.
template <typename R>
__device__ __forceinline__ void apply_g5(cpx<R> s[12]) {
#pragma unroll
    for (int c = 0; c < 6; c++) s[c] = -s[c];
}

}  // namespace ovl

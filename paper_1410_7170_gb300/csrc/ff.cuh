// Float-float arithmetic: a real number carried as the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2 (about 48 significant bits, unit roundoff ~2^-47),
// computed entirely on the FP32 pipes.
//
// Why: GB300 runs FP64 at 1/64 of its FP32 rate (about 2 FP64 FMAs per clock per SM), so
// the Wilson stencil in FP64 is bound by the FP64 pipes at a tenth of the memory
// bandwidth. The sign applications that need more than FP32 accuracy (outer D_N products
// to ~1e-10) run in this arithmetic instead: each float-float operation costs 7-15 FP32
// instructions, a quarter of the time of the FP64 instruction it replaces, and keeps
// rounding errors near 1e-14 relative, far below the 1e-10 the products need.
//
// The building blocks are error-free transformations of FP32 operations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error e, a + b = s + e;
//   Fast2Sum (Dekker 1971): the same for |a| >= |b| in three operations;
//   TwoProduct by FMA: p = fl(a b), e = fma(a, b, -p) is exact, a b = p + e.
// Every operation below uses the _rn intrinsics so the compiler can neither contract an
// addition into a fused multiply-add nor reorder the operations (either would destroy the
// error terms). Products and sums follow the "sloppy" double-single forms: the cross
// terms hi*lo are added in FP32, and the error is bounded relative to the magnitudes of
// the operands (not of the result), which is what the normwise error of a stencil or a
// Krylov recurrence needs.
#pragma once
#include "common.cuh"

namespace ovl {

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr ff(float h) : hi(h), lo(0.f) {}
    __host__ __device__ explicit constexpr ff(int h) : hi((float)h), lo(0.f) {}
    // split of an FP64 value: hi = fl32(d), lo = fl32(d - hi) (d - hi is exact in FP64; lo keeps
    // its leading 24 bits, so hi + lo equals d to about 2^-48 relative)
    __host__ __device__ explicit ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
    return ff(s, e);
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
// a b + c with one renormalisation
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const ff s = ff_two_sum(p, c.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// Storage word of one complex number in float-float: (re.hi, re.lo, im.hi, im.lo), 16 bytes,
// the same size and word layout as an FP64 complex (double2), so the FP64 even-odd layouts
// carry over word for word:
//   float-float spinor: ffw [p][12 spin-colour][Vh]        (192 B per site)
//   float-float link:   ffw [p][mu][9][Vh]   all 18 reals of -1/2 U_mu(x)
struct __align__(16) ffw {
    float rh, rl, ih, il;
};

__device__ __forceinline__ cpx<ff> ffw_get(const float4 v) { return cpx<ff>{ff(v.x, v.y), ff(v.z, v.w)}; }
__device__ __forceinline__ float4 ffw_put(const cpx<ff> &c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }

template <typename R>
__device__ __forceinline__ void load_spinor(const ffw *__restrict__ f, int Vh, int p, int i, cpx<R> s[12]) {
    static_assert(sizeof(R) == sizeof(ff), "float-float storage is read as float-float");
    const float4 *b = reinterpret_cast<const float4 *>(f) + (size_t)p * 12 * Vh + i;
#pragma unroll
    for (int c = 0; c < 12; c++) s[c] = ffw_get(__ldg(b + (size_t)c * Vh));
}
template <typename R>
__device__ __forceinline__ void store_spinor(ffw *__restrict__ f, int Vh, int p, int i, const cpx<R> s[12]) {
    float4 *b = reinterpret_cast<float4 *>(f) + (size_t)p * 12 * Vh + i;
#pragma unroll
    for (int c = 0; c < 12; c++) b[(size_t)c * Vh] = ffw_put(s[c]);
}
template <typename R>
__device__ __forceinline__ void load_link(const ffw *__restrict__ g, int Vh, int p, int mu, int i, cpx<R> u[3][3]) {
    const float4 *b = reinterpret_cast<const float4 *>(g) + ((size_t)(p * 4 + mu) * kLink64Words) * Vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) u[c / 3][c % 3] = ffw_get(__ldg(b + (size_t)c * Vh));
}

}  // namespace ovl

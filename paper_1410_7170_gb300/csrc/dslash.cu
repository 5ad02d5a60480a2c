// Layout conversion and the Wilson-Dirac stencil kernels (Eq. Wilson-Dirac).
#include "internal.h"
#include "reduce.cuh"
#include "wilson_quad.cuh"
#include "wilson_site.cuh"

#include <algorithm>
#include <atomic>

namespace ovl {

static std::atomic<long> g_launches{0};
static thread_local bool g_counting = true;
void count_launches(long n) {
    if (g_counting) g_launches.fetch_add(n, std::memory_order_relaxed);
}
long launches_total() { return g_launches.load(std::memory_order_relaxed); }
void set_launch_counting(bool on) { g_counting = on; }

int device_sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

// ------------------------------------------------------------------ gauge upload
// One thread per (site, mu): SU(3) check, then -1/2 U in both precisions (FP32: rows 0 and 1).
__global__ void k_pack_gauge(Geom g, const double2 *__restrict__ lex, double2 *u64, float4 *u32, int *bad,
                             double tol) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)g.V * 4) return;
    const int s = (int)(t >> 2), mu = (int)(t & 3);
    cpx<double> u[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            double2 v = lex[(size_t)t * 9 + a * 3 + b];
            u[a][b] = cpx<double>{v.x, v.y};
        }
    // unitarity: max |(U U^H - I)_ab|; det U = 1
    double err = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            cpx<double> d = cmul_conj(u[b][0], u[a][0]) + cmul_conj(u[b][1], u[a][1]) + cmul_conj(u[b][2], u[a][2]);
            if (a == b) d.re -= 1.0;
            err = fmax(err, sqrt(norm2(d)));
        }
    cpx<double> det = u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                      u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                      u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]);
    det.re -= 1.0;
    err = fmax(err, sqrt(norm2(det)));
    if (!(err <= tol)) atomicExch(bad, 1);   // also catches NaN
    int x[4];
    int r = s;
    x[3] = r % g.L[3]; r /= g.L[3];
    x[2] = r % g.L[2]; r /= g.L[2];
    x[1] = r % g.L[1]; x[0] = r / g.L[1];
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1, i = s >> 1;
    // stored as kLinkScale U (the hopping term's -1/2 folded in)
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) u[a][b] = kLinkScale * u[a][b];
    double2 *d64 = u64 + ((size_t)(p * 4 + mu) * kLink64Words) * g.Vh + i;
#pragma unroll
    for (int c = 0; c < 9; c++) d64[(size_t)c * g.Vh] = make_double2(u[c / 3][c % 3].re, u[c / 3][c % 3].im);
    float4 *d32 = u32 + ((size_t)(p * 4 + mu) * 3) * g.Vh + i;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cpx<double> e0 = u[(2 * c) / 3][(2 * c) % 3], e1 = u[(2 * c + 1) / 3][(2 * c + 1) % 3];
        d32[(size_t)c * g.Vh] = make_float4((float)e0.re, (float)e0.im, (float)e1.re, (float)e1.im);
    }
}

cudaError_t pack_gauge(const Geom &g, const double *lex, double2 *u64, float4 *u32, int *bad, double tol,
                       cudaStream_t st) {
    k_pack_gauge<<<plain_grid((long)g.V * 4), kBlock, 0, st>>>(g, (const double2 *)lex, u64, u32, bad, tol);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ spinor layout
__device__ __forceinline__ void lex_to_eo(const Geom &g, int s, int &p, int &i) {
    int r = s;
    int x3 = r % g.L[3]; r /= g.L[3];
    int x2 = r % g.L[2]; r /= g.L[2];
    int x1 = r % g.L[1];
    int x0 = r / g.L[1];
    p = (x0 + x1 + x2 + x3) & 1;
    i = s >> 1;
}

__global__ void k_pack_spinor_f64(Geom g, double2 *dst, const double2 *__restrict__ lex) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int p, i;
    lex_to_eo(g, s, p, i);
    cpx<double> v[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
        double2 e = lex[(size_t)s * 12 + c];
        v[c] = cpx<double>{e.x, e.y};
    }
    store_spinor<double>(dst, g.Vh, p, i, v);
}

__global__ void k_unpack_spinor_f64(Geom g, double2 *lex, const double2 *__restrict__ src) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int p, i;
    lex_to_eo(g, s, p, i);
    cpx<double> v[12];
    load_spinor<double>(src, g.Vh, p, i, v);
#pragma unroll
    for (int c = 0; c < 12; c++) lex[(size_t)s * 12 + c] = make_double2(v[c].re, v[c].im);
}

cudaError_t pack_spinor_f64(const Geom &g, double2 *dst, const double *lex, cudaStream_t st) {
    k_pack_spinor_f64<<<plain_grid(g.V), kBlock, 0, st>>>(g, dst, (const double2 *)lex);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t unpack_spinor_f64(const Geom &g, double *lex, const double2 *src, cudaStream_t st) {
    k_unpack_spinor_f64<<<plain_grid(g.V), kBlock, 0, st>>>(g, (double2 *)lex, src);
    count_launches(1);
    return cudaGetLastError();
}

// FP64 <-> FP32 even-odd spinors (double2 [p][12][Vh] <-> float4 [p][6][Vh])
__global__ void k_spinor_d2f(Geom g, const double2 *__restrict__ a, float4 *__restrict__ b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.V) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    cpx<float> v[12];
    load_spinor<float>(a, g.Vh, p, i, v);
    store_spinor<float>(b, g.Vh, p, i, v);
}
__global__ void k_spinor_f2d(Geom g, const float4 *__restrict__ a, double2 *__restrict__ b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.V) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    cpx<double> v[12];
    load_spinor<double>(a, g.Vh, p, i, v);
    store_spinor<double>(b, g.Vh, p, i, v);
}
cudaError_t spinor_d2f(const Geom &g, const double2 *a, float4 *b, cudaStream_t st) {
    k_spinor_d2f<<<plain_grid(g.V), kBlock, 0, st>>>(g, a, b);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t spinor_f2d(const Geom &g, const float4 *a, double2 *b, cudaStream_t st) {
    k_spinor_f2d<<<plain_grid(g.V), kBlock, 0, st>>>(g, a, b);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ stencil
// out = a [g5] D_W(m0) in + b z, one thread per site of the full lattice
// (threads [0, Vh) even sites, [Vh, V) odd sites).
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_wilson(Geom g, const LT *__restrict__ U, const ST *__restrict__ in,
                                                   ST *__restrict__ out, R m4, int g5, R a,
                                                   const ST *z, R b, int spb) {
    const int t = blockIdx.x * spb + threadIdx.x;
    if (threadIdx.x >= spb || t >= g.V) return;
    int p, i;
    site_of_thread(t, p, i);
    cpx<R> hop[12], own[12], res[12];
    wilson_hop<R>(g, U, in, p, i, hop);
    load_spinor<R>(in, g.Vh, p, i, own);
    wilson_combine<R>(m4, own, hop, res);
    if (g5) apply_g5(res);
    if (z) {
        cpx<R> zz[12];
        load_spinor<R>(z, g.Vh, p, i, zz);
#pragma unroll
        for (int c = 0; c < 12; c++) res[c] = a * res[c] + b * zz[c];
    } else {
#pragma unroll
        for (int c = 0; c < 12; c++) res[c] = a * res[c];
    }
    store_spinor<R>(out, g.Vh, p, i, res);
}

// Same with four threads per site (thread q of a quad owns direction mu = q and the
// storage words j with j % 4 == q of the output).
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_wilson4(Geom g, const LT *__restrict__ U, const ST *__restrict__ in,
                                                    ST *__restrict__ out, R m4, int g5, R a, const ST *z, R b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0 = t >> 2, q = t & 3;
    const int s = s0 < g.V ? s0 : g.V - 1;   // quads past the end compute a copy, store nothing
    int p, i;
    site_of_thread(s, p, i);
    cpx<R> acc[12];
    wilson_hop_dir<R>(g, U, in, p, i, q, acc);
    quad_allreduce(acc);
    if (s0 >= g.V) return;
    using C = Chunk<ST>;
#pragma unroll
    for (int j = 0; j < C::NC; j++) {
        if ((j & 3) != q) continue;
        cpx<R> own[C::CPC], res[C::CPC];
        C::template load<R>(in, g.Vh, p, i, j, own);
#pragma unroll
        for (int e = 0; e < C::CPC; e++) {
            const int cix = j * C::CPC + e;
            res[e] = m4 * own[e] + acc[cix];
            if (g5 && cix < 6) res[e] = -res[e];
            res[e] = a * res[e];
        }
        if (z) {
            cpx<R> zz[C::CPC];
            C::template load<R>(z, g.Vh, p, i, j, zz);
#pragma unroll
            for (int e = 0; e < C::CPC; e++) res[e] = res[e] + b * zz[e];
        }
        C::template store<R>(out, g.Vh, p, i, j, res);
    }
}

cudaError_t wilson_f64(const Geom &g, const double2 *U, const double2 *in, double2 *out, double m0, int g5,
                       double a, const double2 *z, double b, cudaStream_t st) {
    if (g.tps64 == 4)
        k_wilson4<double, double2, double2><<<plain_grid(4L * g.V), kBlock, 0, st>>>(g, U, in, out, m0 + 4.0, g5,
                                                                                     a, z, b);
    else {
        const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<double>::value, 1 << 30);
        k_wilson<double, double2, double2><<<ls.grid, ls.block, 0, st>>>(g, U, in, out, m0 + 4.0, g5, a, z, b,
                                                                         ls.spb);
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t wilson_f32(const Geom &g, const float4 *U, const float4 *in, float4 *out, float m0, int g5,
                       float a, const float4 *z, float b, cudaStream_t st) {
    if (g.tps32 == 4)
        k_wilson4<float, float4, float4><<<plain_grid(4L * g.V), kBlock, 0, st>>>(g, U, in, out, m0 + 4.0f, g5, a,
                                                                                  z, b);
    else {
        const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<float>::value, 1 << 30);
        k_wilson<float, float4, float4><<<ls.grid, ls.block, 0, st>>>(g, U, in, out, m0 + 4.0f, g5, a, z, b,
                                                                      ls.spb);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t wilson_ff(const Geom &g, const ffw *U, const ffw *in, ffw *out, double m0, int g5, double a,
                      const ffw *z, double b, cudaStream_t st) {
    const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<ff>::value, 1 << 30);
    k_wilson<ff, ffw, ffw><<<ls.grid, ls.block, 0, st>>>(g, U, in, out, ff(m0 + 4.0), g5, ff(a), z, ff(b), ls.spb);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ 16-bit stencil
// out = D_W(m0) in with 16-bit links and 16-bit spinors (FP16 with a per-site scale, or
// BF16), arithmetic in FP32: per site 4 x 24 B of links and the input and output spinors
// (52 B each in FP16, 48 B in BF16) are the algorithmic traffic, about half of the FP32
// stencil's 384 B.
template <typename LT, typename SIn, typename SOut>
__global__ void __launch_bounds__(kBlock, 2) k_wilson16(Geom g, const LT *__restrict__ U, SIn in, SOut out, float m4,
                                                      int spb) {
    const int t = blockIdx.x * spb + threadIdx.x;
    if (threadIdx.x >= spb || t >= g.V) return;
    int p, i;
    site_of_thread(t, p, i);
    cpx<float> hop[12], own[12], res[12];
    wilson_hop<float>(g, U, in, p, i, hop);
    load_spinor<float>(in, g.Vh, p, i, own);
    wilson_combine<float>(m4, own, hop, res);
    store_spinor<float>(out, g.Vh, p, i, res);
}

// FP32 links (rows 0 and 1, float4 [p][mu][3][Vh]) -> 16-bit links (uint2 [p][mu][3][Vh]):
// every float4 word becomes one 8-byte word.
template <typename L16>
__global__ void k_link_to16(const float4 *__restrict__ u32, L16 *u16, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const float4 v = u32[k];
        reinterpret_cast<uint2 *>(u16)[k] = make_uint2(pack16(u16, v.x, v.y), pack16(u16, v.z, v.w));
    }
}
// FP32 even-odd spinor <-> FP16 (per-site scale) or BF16 even-odd spinor
template <typename S16>
__global__ void k_spinor_f2h(Geom g, const float4 *__restrict__ a, S16 b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.V) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    cpx<float> v[12];
    load_spinor<float>(a, g.Vh, p, i, v);
    store_spinor<float>(b, g.Vh, p, i, v);
}
template <typename S16C>
__global__ void k_spinor_h2f(Geom g, S16C a, float4 *__restrict__ b) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.V) return;
    const int p = t >= g.Vh, i = t - p * g.Vh;
    cpx<float> v[12];
    load_spinor<float>(a, g.Vh, p, i, v);
    store_spinor<float>(b, g.Vh, p, i, v);
}

cudaError_t links_to16(const Geom &g, const float4 *u32, void *u16, bool bf16, cudaStream_t st) {
    const long n = (long)g.V * 4 * 3;
    const int grid = (int)std::min<long>((n + kBlock - 1) / kBlock, 16L * g.nsm);
    if (bf16) k_link_to16<LinkB><<<grid, kBlock, 0, st>>>(u32, (LinkB *)u16, n);
    else k_link_to16<LinkH><<<grid, kBlock, 0, st>>>(u32, (LinkH *)u16, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t spinor_f2h(const Geom &g, const float4 *a, uint4 *v, float *norm, bool bf16, cudaStream_t st) {
    if (bf16) k_spinor_f2h<Bf16Spinor><<<plain_grid(g.V), kBlock, 0, st>>>(g, a, Bf16Spinor{v});
    else k_spinor_f2h<HalfSpinor><<<plain_grid(g.V), kBlock, 0, st>>>(g, a, HalfSpinor{v, norm});
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t spinor_h2f(const Geom &g, const uint4 *v, const float *norm, float4 *b, bool bf16, cudaStream_t st) {
    if (bf16) k_spinor_h2f<Bf16SpinorC><<<plain_grid(g.V), kBlock, 0, st>>>(g, Bf16SpinorC{v}, b);
    else k_spinor_h2f<HalfSpinorC><<<plain_grid(g.V), kBlock, 0, st>>>(g, HalfSpinorC{v, norm}, b);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t wilson_16(const Geom &g, const void *u16, const uint4 *in, const float *in_norm, uint4 *out, float *out_norm,
                      float m0, bool bf16, cudaStream_t st) {
    const LaunchShape ls = balanced_shape(g.V, g.nsm, 2, 1 << 30);
    if (bf16)
        k_wilson16<LinkB, Bf16SpinorC, Bf16Spinor><<<ls.grid, ls.block, 0, st>>>(
            g, (const LinkB *)u16, Bf16SpinorC{in}, Bf16Spinor{out}, m0 + 4.f, ls.spb);
    else
        k_wilson16<LinkH, HalfSpinorC, HalfSpinor><<<ls.grid, ls.block, 0, st>>>(
            g, (const LinkH *)u16, HalfSpinorC{in, in_norm}, HalfSpinor{out, out_norm}, m0 + 4.f, ls.spb);
    count_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ float-float conversion
// double2 word k <-> ffw word k: hi = fl32(x), lo = fl32(x - hi) per real; back, hi + lo in FP64.
__global__ void k_d2ff(const double2 *__restrict__ x, ffw *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const double2 v = x[k];
        const ff re(v.x), im(v.y);
        reinterpret_cast<float4 *>(y)[k] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}
__global__ void k_ff2d(const ffw *__restrict__ x, double2 *__restrict__ y, long n) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(x)[k];
        y[k] = make_double2(ff(v.x, v.y).to_double(), ff(v.z, v.w).to_double());
    }
}
static int conv_grid(long n) {
    long b = (n + kBlock - 1) / kBlock;
    const long cap = 16L * device_sm_count();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}
cudaError_t dev_d2ff(const double2 *x, ffw *y, long n, cudaStream_t st) {
    k_d2ff<<<conv_grid(n), kBlock, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t dev_ff2d(const ffw *x, double2 *y, long n, cudaStream_t st) {
    k_ff2d<<<conv_grid(n), kBlock, 0, st>>>(x, y, n);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace ovl

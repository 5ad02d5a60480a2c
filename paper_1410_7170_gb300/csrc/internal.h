// Internal interfaces between the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>

#include "common.cuh"
#include "ff.cuh"

namespace ovl {

constexpr int kMaxPoles = 64;
constexpr int kBlock = 256;             // threads per block of site-parallel kernels
constexpr int kMaxRedBlocks = 4096;     // cap on blocks of a reducing kernel (grid-stride beyond)
constexpr int kMaxRedValues = 4;        // doubles reduced by one kernel

// Scratch of the deterministic two-level reductions: per-block partial sums, and
// a counter the last finishing block uses to find that it is last.
struct RedScratch {
    double *partials;      // [kMaxRedValues][kMaxRedBlocks]
    unsigned *counter;     // one word, zero between launches
};

// Minimum resident blocks per SM requested from the compiler: the FP64 stencils are
// held to 128 registers so two 256-thread blocks fit on an SM (one wave of 256 blocks
// at 16^4 on 152 SMs).
template <typename R> struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };
template <> struct MinBlocks<float> { static constexpr int value = 2; };
template <> struct MinBlocks<ff> { static constexpr int value = 2; };

// SMs of the current device (queried once per device and cached).
int device_sm_count();

// Blocks of a grid-striding reduction over n_threads elements: enough to fill every SM a
// few times, few enough that the per-block partials and the arrival counter stay cheap.
inline int red_grid(long n_threads) {
    long b = (n_threads + kBlock - 1) / kBlock;
    const long cap = 4L * device_sm_count();
    if (b > cap) b = cap;
    if (b > kMaxRedBlocks) b = kMaxRedBlocks;
    if (b < 1) b = 1;
    return (int)b;
}
// Launch shape for a site-parallel kernel over n sites: the block count is a multiple of
// nsm * per_sm (every SM holds the same number of blocks in every wave), each block owns
// spb consecutive sites (thread t < spb of block b handles site b * spb + t, striding by
// grid * spb), and the block size is spb rounded up to whole warps.
struct LaunchShape {
    int grid, block, spb;
};
inline LaunchShape balanced_shape(long n, int nsm, int per_sm, int max_blocks) {
    if (nsm <= 0) nsm = 1;
    const long slots = (long)nsm * per_sm;
    long waves = (n + slots * kBlock - 1) / (slots * kBlock);
    if (waves < 1) waves = 1;
    long nblk = slots * waves;
    if (nblk > max_blocks) nblk = (max_blocks / slots) * slots;
    if (nblk < 1) nblk = 1;
    long spb = (n + nblk - 1) / nblk;
    if (spb > kBlock) spb = kBlock;   // more sites than threads: the kernel strides
    const int T = (int)((spb + 31) / 32 * 32);
    return LaunchShape{(int)nblk, T, (int)spb};
}

inline int plain_grid(long n_threads) {
    long b = (n_threads + kBlock - 1) / kBlock;
    return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- layouts / gauge
// lex: V*4*9 complex doubles [s][mu][a][b]. Writes the FP64 and FP32 12-real copies;
// sets *bad to 1 if some link misses unitarity or det = 1 by more than tol.
cudaError_t pack_gauge(const Geom &g, const double *lex, double2 *u64, float4 *u32, int *bad, double tol,
                       cudaStream_t st);
// lex spinor [s][12] complex doubles <-> internal even-odd layouts
cudaError_t pack_spinor_f64(const Geom &g, double2 *dst, const double *lex, cudaStream_t st);
cudaError_t unpack_spinor_f64(const Geom &g, double *lex, const double2 *src, cudaStream_t st);

// even-odd FP64 <-> FP32 spinor conversion
cudaError_t spinor_d2f(const Geom &g, const double2 *a, float4 *b, cudaStream_t st);
cudaError_t spinor_f2d(const Geom &g, const float4 *a, double2 *b, cudaStream_t st);

// ---------------------------------------------------------------- stencils
// out = a * [gamma5] D_W(m0) in + b * z   (z may be NULL; then b is ignored)
cudaError_t wilson_f64(const Geom &g, const double2 *U, const double2 *in, double2 *out, double m0, int g5,
                       double a, const double2 *z, double b, cudaStream_t st);
cudaError_t wilson_f32(const Geom &g, const float4 *U, const float4 *in, float4 *out, float m0, int g5,
                       float a, const float4 *z, float b, cudaStream_t st);
// float-float stencil (one thread per site); links in the float-float layout of ff.cuh
cudaError_t wilson_ff(const Geom &g, const ffw *U, const ffw *in, ffw *out, double m0, int g5, double a,
                      const ffw *z, double b, cudaStream_t st);
// 16-bit stencil: out = D_W(m0) in with 16-bit links (from links_to16) and 16-bit spinors,
// FP16 with a per-site scale (norm arrays of V floats) or BF16 (norms unused), FP32 arithmetic
cudaError_t links_to16(const Geom &g, const float4 *u32, void *u16, bool bf16, cudaStream_t st);
cudaError_t spinor_f2h(const Geom &g, const float4 *a, uint4 *v, float *norm, bool bf16, cudaStream_t st);
cudaError_t spinor_h2f(const Geom &g, const uint4 *v, const float *norm, float4 *b, bool bf16, cudaStream_t st);
cudaError_t wilson_16(const Geom &g, const void *u16, const uint4 *in, const float *in_norm, uint4 *out, float *out_norm,
                      float m0, bool bf16, cudaStream_t st);
// FP64 <-> float-float conversion of n complex words (double2 <-> ffw, same word order; used
// for even-odd spinors and for the FP64 link array)
cudaError_t dev_d2ff(const double2 *x, ffw *y, long n, cudaStream_t st);
cudaError_t dev_ff2d(const ffw *x, double2 *y, long n, cudaStream_t st);

// ---------------------------------------------------------------- BLAS-1 (flat arrays of n doubles)
// Reductions return through device memory `res` (written by the last block).
cudaError_t dev_norm2(const double *x, long n, double *res, RedScratch rs, cudaStream_t st);
// res[0] = Re <x,y>, res[1] = Im <x,y> (complex interleaved, n doubles = n/2 complex)
cudaError_t dev_cdot(const double *x, const double *y, long n, double *res, RedScratch rs, cudaStream_t st);
// y = a x + b y (real a, b)
cudaError_t dev_axpby(double a, const double *x, double b, double *y, long n, cudaStream_t st);
// y += (ar + i ai) x  (complex, interleaved)
cudaError_t dev_caxpy(double ar, double ai, const double *x, double *y, long n, cudaStream_t st);
// Arnoldi helpers: out[2k..2k+1] = <v_k, w> for k < m (v_k = base + k*stride), deterministic
cudaError_t dev_multidot(const double *base, long stride, int m, const double *w, long n, double *out,
                         double *partials, cudaStream_t st);
// w += sum_k c_k v_k, c complex interleaved in device memory (m <= 128)
cudaError_t dev_multiaxpy(const double *base, long stride, int m, const double *c, double *w, long n,
                          cudaStream_t st);
// float <-> double conversion of flat arrays (same element order)
cudaError_t dev_d2f(const double *x, float *y, long n, cudaStream_t st);
cudaError_t dev_f2d(const float *x, double *y, long n, cudaStream_t st);
// y = a*x + b*y on floats
cudaError_t dev_axpby_f(float a, const float *x, float b, float *y, long n, cudaStream_t st);
cudaError_t dev_norm2_f(const float *x, long n, double *res, RedScratch rs, cudaStream_t st);
cudaError_t dev_cdot_f(const float *x, const float *y, long n, double *res, RedScratch rs, cudaStream_t st);
// multi-dot / multi-axpy with float vectors (accumulation in double)
cudaError_t dev_multidot_f(const float *base, long stride, int m, const float *w, long n, double *out,
                           double *partials, cudaStream_t st);
// out[0 .. 2m-1] = <base_j, w> (complex), out[2m] = ||w||^2, out[2m+1] = 0, in one pass.
cudaError_t dev_multidot_norm_f(const float *base, long stride, int m, const float *w, long n, double *out,
                                double *partials, cudaStream_t st);
// out = scale (w - sum_j h_j base_j), h = the complex dots of dev_multidot_norm_f (device).
cudaError_t dev_orth_scale_f(const float *base, long stride, int m, const double *h, double scale, const float *w,
                             float *out, long n, cudaStream_t st);
cudaError_t dev_multiaxpy_f(const float *base, long stride, int m, const double *c, float *w, long n,
                            cudaStream_t st);
// x[k] = seeded pseudo-random values in [-1, 1) (a counter hash of k and the seed)
cudaError_t fill_random_f32(float *x, long n, unsigned seed, cudaStream_t st);
// Finite check of a flat array: *flag = 1 if some entry is NaN/Inf.
cudaError_t dev_nonfinite(const double *x, long n, int *flag, cudaStream_t st);

// ---------------------------------------------------------------- multishift CG
// Device-side state of one multishift solve (Q^2 + sigma_l) x_l = b, l < n, with the
// Zolotarev accumulation y = b + sum_l w_l x_l. sigma[0] is the base (smallest) shift.
struct MsState {
    int n;                     // shifts
    int iter;                  // iterations done
    int done;                  // 1: all shifts converged (kernels then do nothing)
    int status;                // 0 ok, 1 breakdown / non-finite scalar
    double bb;                 // ||b||^2
    double rr;                 // ||r_k||^2 (base residual)
    double pp;                 // ||p_0||^2 by the recurrence ||p_k||^2 = ||r_k||^2 + b_{k-1}^2 ||p_{k-1}||^2
    double alpha, alpha_prev, beta_prev;
    double tol;                // target relative accuracy of the rational function
    double sigma[kMaxPoles];   // shifts
    double w[kMaxPoles];       // weights of x_l in y
    double crit[kMaxPoles];    // drop shift l when crit_l * |zeta_l| * ||r|| <= tol * ||b||
    double zeta[kMaxPoles], zeta_prev[kMaxPoles];
    double alpha_l[kMaxPoles], beta_l[kMaxPoles];   // this iteration's coefficients of the rescaled directions
                                                    // (y += w_l alpha_l p~_l, p~_l = r + beta_l p~_l)
    int active[kMaxPoles];
    int *hist;                 // optional: hist[k] = shifts updated in iteration k (instrumentation)
    int hist_cap;
};

// Workspace vectors of a multishift solve, in storage type ST.
template <typename ST>
struct MsVectors {
    ST *r;       // base residual
    ST *t;       // Q p_0
    ST *y;       // accumulated rational function argument
    ST *p;       // n search directions, p[l] at p + l * stride
    ST *r2;      // FP32 only: second residual buffer of the fused iteration (r_k in r for even k, r2 odd)
    long stride; // elements of ST per vector
};

// Half-precision variant of the FP32 multishift vectors: p_0 (the base direction, which
// drives the Krylov process), r, t and y stay FP32; the shifted directions p_l, l >= 1,
// are stored as FP16 scaled by a per-site FP32 norm (see HalfSpinor).
struct MsVectorsH {
    float4 *r, *t, *y, *p0;
    uint4 *ph;          // p_l for l >= 1 at ph + (l - 1) * words_h
    float *pn;          // their per-site norms at pn + (l - 1) * V
    long words;         // float4 words per FP32 vector (6 V)
    long words_h;       // uint4 words per FP16 vector (3 V)
};

// One multishift iteration = three launches (Q p, residual update, shift updates).
// ev (optional, 4 events): recorded before/between/after the first three launches;
// ev_flags is passed to cudaEventRecordWithFlags (cudaEventRecordExternal inside graphs).
cudaError_t ms_init_f64(const Geom &g, int n, MsState *s, MsVectors<double2> v, const double2 *b, RedScratch rs,
                        cudaStream_t st);
cudaError_t ms_iter_f64(const Geom &g, const double2 *U, double m0, MsState *s, MsVectors<double2> v,
                        RedScratch rs, cudaStream_t st, cudaEvent_t *ev = nullptr, unsigned ev_flags = 0);
cudaError_t ms_init_f32(const Geom &g, int n, MsState *s, MsVectors<float4> v, const float4 *b, RedScratch rs,
                        cudaStream_t st);
cudaError_t ms_iter_f32(const Geom &g, const float4 *U, float m0, MsState *s, MsVectors<float4> v,
                        RedScratch rs, cudaStream_t st, cudaEvent_t *ev = nullptr, unsigned ev_flags = 0);
cudaError_t ms_init_half(const Geom &g, int n, MsState *s, MsVectorsH v, const float4 *b, RedScratch rs, bool bf16,
                         cudaStream_t st);
// float-float multishift (the FP64-accuracy sign on the FP32 pipes)
cudaError_t ms_init_ff(const Geom &g, int n, MsState *s, MsVectors<ffw> v, const ffw *b, RedScratch rs,
                       cudaStream_t st);
cudaError_t ms_iter_ff(const Geom &g, const ffw *U, double m0, MsState *s, MsVectors<ffw> v, RedScratch rs,
                       cudaStream_t st, cudaEvent_t *ev = nullptr, unsigned ev_flags = 0);
cudaError_t ms_iter_half(const Geom &g, const float4 *U, float m0, MsState *s, MsVectorsH v, RedScratch rs, bool bf16,
                         cudaStream_t st, cudaEvent_t *ev = nullptr, unsigned ev_flags = 0);

// ---------------------------------------------------------------- several right-hand sides
constexpr int kMaxBatch = 12;   // right-hand sides per batch (threads 32 x nrhs per block)

// out_y = a [gamma5] D_W(m0) in_y + b z_y for y < nrhs; vectors `stride` storage words apart.
cudaError_t wilson_batch_f64(const Geom &g, const double2 *U, const double2 *in, double2 *out, long stride, int nrhs,
                             double m0, int g5, double a, const double2 *z, double b, cudaStream_t st);
cudaError_t wilson_batch_f32(const Geom &g, const float4 *U, const float4 *in, float4 *out, long stride, int nrhs,
                             float m0, int g5, float a, const float4 *z, float b, cudaStream_t st);

// Batched multishift vectors: per right-hand side y, r/t/y at base + y * stride and its
// npole directions at p + (y * npole + l) * stride.
template <typename ST>
struct MsBatch {
    ST *r, *t, *y, *p;
    long stride;
};
// One state per right-hand side (st[y]); partial sums need nrhs * 2 * kMaxRedBlocks doubles;
// counters: nrhs words, zero between launches.
cudaError_t msb_init_f64(const Geom &g, int nrhs, int npole, MsState *st, MsBatch<double2> v, const double2 *b,
                         RedScratch rs, cudaStream_t s);
cudaError_t msb_init_f32(const Geom &g, int nrhs, int npole, MsState *st, MsBatch<float4> v, const float4 *b,
                         RedScratch rs, cudaStream_t s);
cudaError_t msb_iter_f64(const Geom &g, const double2 *U, double m0, int nrhs, int npole, MsState *st,
                         MsBatch<double2> v, RedScratch rs, unsigned *counters, cudaStream_t s);
cudaError_t msb_iter_f32(const Geom &g, const float4 *U, float m0, int nrhs, int npole, MsState *st,
                         MsBatch<float4> v, RedScratch rs, unsigned *counters, cudaStream_t s);

// Process-wide count of kernel launches issued by the library (instrumentation).
void count_launches(long n);
long launches_total();
void set_launch_counting(bool on);

// Message returned by ovl_last_error(NULL) on the calling thread.
void set_thread_error(const std::string &msg);

// ---------------------------------------------------------------- host Zolotarev
int zolotarev_host(double k, int n, double *d0, double *a, double *c, double *delta);

// Eigenvalues (ascending) and eigenvectors (columns of Z, row-major) of a small complex
// Hermitian matrix A (row-major, overwritten), by Householder tridiagonalisation and implicit QR; 0 on convergence.
int hermitian_eig(int n, std::complex<double> *A, double *w, std::complex<double> *Z);

}  // namespace ovl

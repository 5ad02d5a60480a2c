// Multishift conjugate gradients for the Zolotarev partial fractions of sign(Q).
//
// The n shifted systems (Q^2 + sigma_l) x_l = b share one Krylov space. The base
// system (smallest shift sigma_0) runs plain CG; shift l keeps its own direction
// p_l and scalars from the shifted-CG recurrences (Jegerlehner, hep-lat/9612014;
// Frommer, "BiCGStab(l) for families of shifted linear systems", 2003):
//
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
//                ( a_k b_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} a_{k-1} (1 + (sigma_l - sigma_0) a_k) )
//   a^l_k = a_k zeta_{k+1}/zeta_k,   b^l_k = b_k (zeta_{k+1}/zeta_k)^2
//   x_l += a^l_k p_l,   p_l = zeta_{k+1} r_{k+1} + b^l_k p_l,   r^l = zeta r.
//
// x_l is never stored: the rational function needs only y = b + sum_l w_l x_l, so
// each iteration adds w_l a^l_k p_l to y. Shift l is dropped once its residual
// bound crit_l |zeta_l| ||r|| falls below tol ||b||.
//
// The directions are stored rescaled, p~_l = p_l / zeta_l (p~_0 = p_0, zeta_0 = 1; p~_l
// stays of the size of r). The updates then take one fused multiply-add per real each,
// against three instructions for the unscaled form (the FP64 shift update is bound by
// the FP64 pipes):
//   y += (w_l a_k zeta_{k+1}) p~_l,   p~_l = r_{k+1} + (b_k zeta_{k+1}/zeta_k) p~_l.
//
// One iteration = three kernels, all scalars stay on the device:
//   ms_q:      t = Q p_0 (stencil with gamma5),       reduce ||t||^2 -> alpha
//   ms_r:      r -= alpha (gamma5 D_W t + sigma_0 p_0), reduce ||r||^2 -> beta, shift scalars
//   ms_shifts: y += sum_l w~_l p~_l ; p~_l = r + b~_l p~_l   (pure streaming)
// The FP32 iteration with one thread per site instead updates the shifted directions one
// iteration late, inside ms_r, where their memory traffic overlaps the stencil's waits:
//   ms_q (+ zeta):  t = Q p_0, alpha_k, and zeta_{k+1} of every shift (it needs only alpha_k
//                   and the previous iteration's scalars)
//   ms_rf:          r_{k+1} = r_k - alpha_k (Q t + sigma_0 p_0); at the same site
//                   p~_l(k) = r_k + b^l_{k-1} p~_l(k-1) (l >= 1) and y += w_l alpha^l_k p~_l(k)
//                   (l >= 0); reduce ||r_{k+1}||^2 -> beta_k, b^l_k, dropped shifts
//   ms_p0:          p_0 = r_{k+1} + beta_k p_0 (the stencil of the next ms_q reads it)
// r alternates between two buffers (r_k in r for even k, in r2 for odd k), so the shift
// updates of ms_rf can read r_k at any point of the kernel.
// The arithmetic of each update is the same as in the three-kernel form; only p~_l(k) is
// formed in iteration k instead of at the end of iteration k-1. In ms_rf odd warps stream
// their shift updates before their stencil and even warps after it, so that on every SM
// some warps stream while the others gather. Measured at 16^4 the FP32 iteration falls from
// 49 to 47 us; the float-float one rose from 147 to 171 us (its shift updates are float-float
// arithmetic on a kernel already bound by arithmetic), so FP64 and float-float keep the
// three-kernel form.
// (p_0, Q^2 p_0) = ||Q p_0||^2 because Q is Hermitian (Eq. gamma_5_symmetry).
// After convergence (state->done) every kernel returns at once, so a fixed number
// of iterations can be queued or captured in a CUDA graph without host round trips.
#include <math.h>

#include "internal.h"
#include "reduce.cuh"
#include "wilson_quad.cuh"
#include "wilson_site.cuh"

namespace ovl {

namespace {

// alpha = (r, r) / (p, (Q^2 + sigma_0) p) with (p, Q^2 p) = ||Q p||^2 (v[0], reduced by ms_q)
// and ||p||^2 from the scalar recurrence ||p_k||^2 = ||r_k||^2 + beta^2 ||p_{k-1}||^2, which
// holds because r_k is orthogonal to p_{k-1} in CG; this spares ms_q a second reduction.
struct AlphaFin {
    MsState *s;
    __device__ void operator()(const double *v) const {
        const double pAp = v[0] + s->sigma[0] * s->pp;
        const double a = s->rr / pAp;
        if (!(pAp > 0.0) || !isfinite(a)) {
            s->status = 1;
            s->done = 1;
            return;
        }
        s->alpha = a;
    }
};

// Shift scalars after the residual update, one warp: lane j handles shifts j, j+32.
struct ShiftFin {
    MsState *s;
    __device__ void operator()(const double *v, int lane) const {
        const double rr_new = v[0];
        const double a = s->alpha, ap = s->alpha_prev, bp = s->beta_prev, rr_old = s->rr;
        const double beta = rr_new / rr_old;
        const int n = s->n;
        if (!isfinite(beta)) {
            if (lane == 0) {
                s->status = 1;
                s->done = 1;
            }
            return;
        }
        const double rnorm = sqrt(rr_new), bnorm = sqrt(s->bb), tolb = s->tol * bnorm;
        int any = 0, nupd = 0;
        for (int l = lane; l < n; l += 32) {
            if (!s->active[l]) {
                s->alpha_l[l] = 0.0;
                continue;
            }
            nupd++;
            double zn;
            if (l == 0) {
                zn = 1.0;
            } else {
                const double z = s->zeta[l], zp = s->zeta_prev[l];
                const double den = a * bp * (zp - z) + zp * ap * (1.0 + (s->sigma[l] - s->sigma[0]) * a);
                zn = (den != 0.0) ? z * zp * ap / den : 0.0;
            }
            const double ratio = (s->zeta[l] != 0.0) ? zn / s->zeta[l] : 0.0;
            // directions stored as p~_l = p_l / zeta_l (see the header): y += w_l a zeta_new p~_l,
            // p~_l = r + b ratio p~_l
            s->alpha_l[l] = a * zn;
            s->beta_l[l] = beta * ratio;
            s->zeta_prev[l] = s->zeta[l];
            s->zeta[l] = zn;
            // residual bound after this iteration's update: drop the shift next time
            if (s->crit[l] * fabs(zn) * rnorm <= tolb) s->active[l] = 2;   // last update
            else any = 1;
        }
        any = __any_sync(0xffffffffu, any);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nupd += __shfl_down_sync(0xffffffffu, nupd, off);
        __syncwarp();
        if (lane == 0) {
            // the base direction p_0 drives the Krylov space: keep it while any shift is live
            if (any && s->active[0] == 2) s->active[0] = 1;
            if (s->hist && s->iter < s->hist_cap) s->hist[s->iter] = nupd;
            s->alpha_prev = a;
            s->beta_prev = beta;
            s->pp = rr_new + beta * beta * s->pp;
            s->rr = rr_new;
            s->iter += 1;
            if (!any) s->done = 2;   // finish this iteration's shift updates, then stop
        }
    }
};

// Fused form, end of ms_q (one warp, lane j handles shifts j, j+32): alpha_k, then for every
// active shift zeta_{k+1} and alpha^l_k = alpha_k zeta_{k+1} (the coefficient of this
// iteration's y update); the base shift has zeta = 1.
struct AlphaFinZ {
    MsState *s;
    __device__ void operator()(const double *v, int lane) const {
        const double pAp = v[0] + s->sigma[0] * s->pp;
        const double a = s->rr / pAp;
        if (!(pAp > 0.0) || !isfinite(a)) {
            if (lane == 0) {
                s->status = 1;
                s->done = 1;
            }
            return;
        }
        const double ap = s->alpha_prev, bp = s->beta_prev;
        for (int l = lane; l < s->n; l += 32) {
            if (!s->active[l]) continue;
            double zn = 1.0;
            if (l > 0) {
                const double z = s->zeta[l], zp = s->zeta_prev[l];
                const double den = a * bp * (zp - z) + zp * ap * (1.0 + (s->sigma[l] - s->sigma[0]) * a);
                zn = (den != 0.0) ? z * zp * ap / den : 0.0;
            }
            s->alpha_l[l] = a * zn;
            s->zeta_prev[l] = s->zeta[l];
            s->zeta[l] = zn;
        }
        __syncwarp();
        if (lane == 0) s->alpha = a;
    }
};

// Fused form, end of ms_rf: beta_k, the next iteration's direction coefficients
// b^l_k = beta_k zeta_{k+1} / zeta_k, and the drop rule on the residual bound after this
// iteration's update (whose y contribution ms_rf has already added, so a dropped shift
// retires at once). The base direction stays while any shift is open.
struct ShiftFinL {
    MsState *s;
    __device__ void operator()(const double *v, int lane) const {
        const double rr_new = v[0];
        const double beta = rr_new / s->rr;
        if (!isfinite(beta)) {
            if (lane == 0) {
                s->status = 1;
                s->done = 1;
            }
            return;
        }
        const double rnorm = sqrt(rr_new), tolb = s->tol * sqrt(s->bb);
        int any = 0, nupd = 0;
        for (int l = lane; l < s->n; l += 32) {
            if (!s->active[l]) continue;
            nupd++;
            const double z = s->zeta[l], zp = s->zeta_prev[l];
            s->beta_l[l] = beta * ((zp != 0.0) ? z / zp : 0.0);
            const bool conv = s->crit[l] * fabs(z) * rnorm <= tolb;
            if (!conv) any = 1;
            else if (l > 0) s->active[l] = 0;
        }
        any = __any_sync(0xffffffffu, any);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nupd += __shfl_down_sync(0xffffffffu, nupd, off);
        __syncwarp();
        if (lane == 0) {
            if (s->hist && s->iter < s->hist_cap) s->hist[s->iter] = nupd;
            s->alpha_prev = s->alpha;
            s->beta_prev = beta;
            s->pp = rr_new + beta * beta * s->pp;
            s->rr = rr_new;
            s->iter += 1;
            if (!any) s->done = 1;
        }
    }
};

// t = gamma5 D_W(m) p0 ; reduce ||t||^2 (Fused: also the shifts' zeta_{k+1}, AlphaFinZ)
template <typename R, typename LT, typename ST, bool Fused>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_ms_q(Geom g, const LT *__restrict__ U, R m4, MsState *s,
                                                 const ST *__restrict__ p0, ST *__restrict__ t, RedScratch rs,
                                                 int spb) {
    if (s->done) return;
    R v[1] = {R(0)};   // per-thread sums in R; FP64 from the warp sums on (grid_reduce)
    const bool lane_has_sites = threadIdx.x < spb;
    for (int k = blockIdx.x * spb + threadIdx.x; lane_has_sites && k < g.V; k += gridDim.x * spb) {
        int p, i;
        site_of_thread(k, p, i);
        cpx<R> hop[12], own[12], res[12];
        wilson_hop<R>(g, U, p0, p, i, hop);
        load_spinor<R>(p0, g.Vh, p, i, own);
        wilson_combine<R>(m4, own, hop, res);
        apply_g5(res);
        store_spinor<R>(t, g.Vh, p, i, res);
        R a0 = R(0);   // per-site sums in the arithmetic type, across sites in FP64
#pragma unroll
        for (int c = 0; c < 12; c++) a0 += norm2(res[c]);
        v[0] += a0;
    }
    if constexpr (Fused) grid_reduce_warp<1>(v, rs, AlphaFinZ{s});
    else grid_reduce<1>(v, rs, AlphaFin{s});
}

// r -= alpha (gamma5 D_W(m) t + sigma0 p0) ; reduce ||r||^2 ; shift scalars
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_ms_r(Geom g, const LT *__restrict__ U, R m4, MsState *s,
                                                 const ST *__restrict__ t, const ST *__restrict__ p0,
                                                 ST *__restrict__ r, RedScratch rs, int spb) {
    if (s->done) return;
    const R alpha = (R)s->alpha, sig0 = (R)s->sigma[0];
    R v[1] = {R(0)};
    const bool lane_has_sites = threadIdx.x < spb;
    for (int k = blockIdx.x * spb + threadIdx.x; lane_has_sites && k < g.V; k += gridDim.x * spb) {
        int p, i;
        site_of_thread(k, p, i);
        cpx<R> hop[12], own[12], res[12], pp[12], rv[12];
        wilson_hop<R>(g, U, t, p, i, hop);
        load_spinor<R>(t, g.Vh, p, i, own);
        wilson_combine<R>(m4, own, hop, res);
        apply_g5(res);
        load_spinor<R>(p0, g.Vh, p, i, pp);
        load_spinor<R>(r, g.Vh, p, i, rv);
        R a0 = R(0);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            rv[c] = rv[c] - alpha * (res[c] + sig0 * pp[c]);
            a0 += norm2(rv[c]);
        }
        v[0] += a0;
        store_spinor<R>(r, g.Vh, p, i, rv);
    }
    grid_reduce_warp<1>(v, rs, ShiftFin{s});
}

// Four-threads-per-site versions (see wilson_quad.cuh). The loops stride by whole
// blocks so every lane of a warp runs the same trip count (the shuffles need all lanes).
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_ms_q4(Geom g, const LT *__restrict__ U, R m4, MsState *s,
                                                  const ST *__restrict__ p0, ST *__restrict__ t, RedScratch rs) {
    if (s->done) return;
    using C = Chunk<ST>;
    R v[1] = {0};
    const long nthr = 4L * g.V;
    for (long base = (long)blockIdx.x * blockDim.x; base < nthr; base += (long)gridDim.x * blockDim.x) {
        const long tt = base + threadIdx.x;
        const int s0 = (int)(tt >> 2), q = (int)(tt & 3);
        const int site = s0 < g.V ? s0 : g.V - 1;
        int p, i;
        site_of_thread(site, p, i);
        cpx<R> acc[12];
        wilson_hop_dir<R>(g, U, p0, p, i, q, acc);
        quad_allreduce(acc);
        if (s0 >= g.V) continue;
#pragma unroll
        for (int j = 0; j < C::NC; j++) {
            if ((j & 3) != q) continue;
            cpx<R> own[C::CPC], res[C::CPC];
            C::template load<R>(p0, g.Vh, p, i, j, own);
            R a0 = 0;
#pragma unroll
            for (int e = 0; e < C::CPC; e++) {
                const int cix = j * C::CPC + e;
                res[e] = m4 * own[e] + acc[cix];
                if (cix < 6) res[e] = -res[e];
                a0 += norm2(res[e]);
            }
            v[0] += a0;
            C::template store<R>(t, g.Vh, p, i, j, res);
        }
    }
    grid_reduce<1>(v, rs, AlphaFin{s});
}

template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_ms_r4(Geom g, const LT *__restrict__ U, R m4, MsState *s,
                                                  const ST *__restrict__ t, const ST *__restrict__ p0,
                                                  ST *__restrict__ r, RedScratch rs) {
    if (s->done) return;
    using C = Chunk<ST>;
    const R alpha = (R)s->alpha, sig0 = (R)s->sigma[0];
    R v[1] = {0};
    const long nthr = 4L * g.V;
    for (long base = (long)blockIdx.x * blockDim.x; base < nthr; base += (long)gridDim.x * blockDim.x) {
        const long tt = base + threadIdx.x;
        const int s0 = (int)(tt >> 2), q = (int)(tt & 3);
        const int site = s0 < g.V ? s0 : g.V - 1;
        int p, i;
        site_of_thread(site, p, i);
        cpx<R> acc[12];
        wilson_hop_dir<R>(g, U, t, p, i, q, acc);
        quad_allreduce(acc);
        if (s0 >= g.V) continue;
#pragma unroll
        for (int j = 0; j < C::NC; j++) {
            if ((j & 3) != q) continue;
            cpx<R> own[C::CPC], pp[C::CPC], rv[C::CPC];
            C::template load<R>(t, g.Vh, p, i, j, own);
            C::template load<R>(p0, g.Vh, p, i, j, pp);
            C::template load<R>(r, g.Vh, p, i, j, rv);
            R a0 = 0;
#pragma unroll
            for (int e = 0; e < C::CPC; e++) {
                const int cix = j * C::CPC + e;
                cpx<R> res = m4 * own[e] + acc[cix];
                if (cix < 6) res = -res;
                rv[e] = rv[e] - alpha * (res + sig0 * pp[e]);
                a0 += norm2(rv[e]);
            }
            v[0] += a0;
            C::template store<R>(r, g.Vh, p, i, j, rv);
        }
    }
    grid_reduce_warp<1>(v, rs, ShiftFin{s});
}

// Elementwise access to a storage word as NR reals.
template <typename ST> struct Word;
// A = arithmetic type of the elementwise updates (the storage precision).
template <> struct Word<double2> {
    static constexpr int N = 2;
    using A = double;
    __device__ static void get(const double2 &w, A *o) { o[0] = w.x; o[1] = w.y; }
    __device__ static double2 put(const A *o) { return make_double2(o[0], o[1]); }
};
template <> struct Word<float4> {
    static constexpr int N = 4;
    using A = float;
    __device__ static void get(const float4 &w, A *o) { o[0] = w.x; o[1] = w.y; o[2] = w.z; o[3] = w.w; }
    __device__ static float4 put(const A *o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
// float-float: one complex number per 16-byte word, (re.hi, re.lo, im.hi, im.lo)
template <> struct Word<ffw> {
    static constexpr int N = 2;
    using A = ff;
    __device__ static void get(const ffw &w, A *o) { o[0] = ff(w.rh, w.rl); o[1] = ff(w.ih, w.il); }
    __device__ static ffw put(const A *o) { return ffw{o[0].hi, o[0].lo, o[1].hi, o[1].lo}; }
};

// y += sum_l w_l a^l p_l ; p_l = zeta_l r + b^l p_l   (words of ST; nw words per vector).
// The active shifts are compacted into a list in shared memory and processed four at
// a time: the four loads of a batch are issued before any store, so each thread keeps
// four independent memory requests in flight.
template <typename ST>
__global__ void __launch_bounds__(kBlock) k_ms_shifts(MsState *s, const ST *__restrict__ r, ST *__restrict__ y,
                                                      ST *__restrict__ P, long stride, long nw, unsigned *counter) {
    using A = typename Word<ST>::A;
    __shared__ A sw[kMaxPoles], sb[kMaxPoles];
    __shared__ int sidx[kMaxPoles];
    __shared__ int sact, sdone;
    if (threadIdx.x == 0) {
        sdone = s->done;
        int na = 0;
        if (sdone != 1)
            for (int l = 0; l < s->n; l++)
                if (s->active[l]) {
                    sidx[na] = l;
                    sw[na] = (A)(s->w[l] * s->alpha_l[l]);
                    sb[na] = (A)s->beta_l[l];
                    na++;
                }
        sact = na;
    }
    __syncthreads();
    if (sdone == 1) return;
    const int na = sact;
    constexpr int N = Word<ST>::N;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (long)gridDim.x * blockDim.x) {
        A rv[N], yv[N];
        Word<ST>::get(r[k], rv);
        Word<ST>::get(y[k], yv);
        for (int a0 = 0; a0 < na; a0 += 4) {
            ST w[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (a0 + u < na) w[u] = P[(long)sidx[a0 + u] * stride + k];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (a0 + u >= na) break;
                A pv[N];
                Word<ST>::get(w[u], pv);
                const A wl = sw[a0 + u], bl = sb[a0 + u];
#pragma unroll
                for (int e = 0; e < N; e++) {
                    yv[e] = fma_r(wl, pv[e], yv[e]);
                    pv[e] = fma_r(bl, pv[e], rv[e]);
                }
                P[(long)sidx[a0 + u] * stride + k] = Word<ST>::put(pv);
            }
        }
        y[k] = Word<ST>::put(yv);
    }
    // the last block retires the shifts that made their final update and ends a finished solve
    if (grid_last_block(counter)) {
        for (int l = threadIdx.x; l < s->n; l += blockDim.x)
            if (s->active[l] == 2) s->active[l] = 0;
        __syncthreads();
        if (threadIdx.x == 0 && s->done == 2) s->done = 1;
    }
}

// Lagged shift updates at site (p, i), word by word: y += wa0 p_0 ; for the active shifts
// l >= 1: p~_l = r_k + b_l p~_l, y += wa_l p~_l.
template <typename ST, typename R>
__device__ __forceinline__ void shift_updates_site(const ST *__restrict__ rk, ST *__restrict__ P, long stride,
                                                   ST *__restrict__ y, int Vh, int p, int i, int na, const int *sidx,
                                                   const R *sw, const R *sb, R sw0) {
    constexpr int N = Word<ST>::N, W = 24 / N;
    constexpr int kB = 2;   // shifts whose words are loaded together
#pragma unroll 2
    for (int w = 0; w < W; w++) {
        const size_t off = ((size_t)p * W + w) * Vh + i;
        R rw[N], yv[N], p0[N];
        Word<ST>::get(rk[off], rw);
        Word<ST>::get(y[off], yv);
        Word<ST>::get(P[off], p0);
#pragma unroll
        for (int e = 0; e < N; e++) yv[e] = fma_r(sw0, p0[e], yv[e]);
        for (int a0 = 0; a0 < na; a0 += kB) {
            ST wv[kB];
#pragma unroll
            for (int u = 0; u < kB; u++)
                if (a0 + u < na) wv[u] = P[(long)sidx[a0 + u] * stride + off];
#pragma unroll
            for (int u = 0; u < kB; u++) {
                if (a0 + u >= na) break;
                R pv[N];
                Word<ST>::get(wv[u], pv);
                const R wl = sw[a0 + u], bl = sb[a0 + u];
#pragma unroll
                for (int e = 0; e < N; e++) {
                    pv[e] = fma_r(bl, pv[e], rw[e]);
                    yv[e] = fma_r(wl, pv[e], yv[e]);
                }
                P[(long)sidx[a0 + u] * stride + off] = Word<ST>::put(pv);
            }
        }
        y[off] = Word<ST>::put(yv);
    }
}

// Fused residual kernel (one thread per site): r_{k+1} = r_k - alpha (gamma5 D_W t + sigma_0 p_0)
// and the lagged shift updates of the same site; reduce ||r_{k+1}||^2 -> ShiftFinL.
// r_k is read from buf[k & 1] and r_{k+1} written to buf[(k + 1) & 1] (buf = {r, r2}), so the
// shift updates can read r_k after the stencil has produced r_{k+1}.
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) k_ms_rf(Geom g, const LT *__restrict__ U, R m4,
                                                                     MsState *s, const ST *__restrict__ t, ST *P,
                                                                     long stride, ST *r, ST *r2, ST *y,
                                                                     RedScratch rs, int spb) {
    __shared__ R sw[kMaxPoles], sb[kMaxPoles];
    __shared__ int sidx[kMaxPoles];
    __shared__ int sact, sdone;
    __shared__ R sw0;
    __shared__ int sodd;
    if (threadIdx.x == 0) {
        sdone = s->done;
        sodd = s->iter & 1;
        int na = 0;
        if (!sdone)
            for (int l = 1; l < s->n; l++)
                if (s->active[l]) {
                    sidx[na] = l;
                    sw[na] = R(s->w[l] * s->alpha_l[l]);
                    sb[na] = R(s->beta_l[l]);
                    na++;
                }
        sact = na;
        sw0 = R(s->w[0] * s->alpha_l[0]);
    }
    __syncthreads();
    if (sdone) return;
    const int na = sact;
    const ST *rin = sodd ? r2 : r;
    ST *rout = sodd ? r : r2;
    const R alpha = R(s->alpha), sig0 = R(s->sigma[0]), w0 = sw0;
    R v[1] = {R(0)};
    const bool shifts_first = (threadIdx.x >> 5) & 1;
    const bool lane_has_sites = threadIdx.x < spb;
    for (int k = blockIdx.x * spb + threadIdx.x; lane_has_sites && k < g.V; k += gridDim.x * spb) {
        int p, i;
        site_of_thread(k, p, i);
        if (shifts_first) shift_updates_site<ST, R>(rin, P, stride, y, g.Vh, p, i, na, sidx, sw, sb, w0);
        {
            cpx<R> hop[12], own[12], res[12], pp[12], rv[12];
            wilson_hop<R>(g, U, t, p, i, hop);
            load_spinor<R>(t, g.Vh, p, i, own);
            wilson_combine<R>(m4, own, hop, res);
            apply_g5(res);
            load_spinor<R>(P, g.Vh, p, i, pp);
            load_spinor<R>(rin, g.Vh, p, i, rv);
            R a0 = R(0);
#pragma unroll
            for (int c = 0; c < 12; c++) {
                rv[c] = rv[c] - alpha * (res[c] + sig0 * pp[c]);
                a0 += norm2(rv[c]);
            }
            v[0] += a0;
            store_spinor<R>(rout, g.Vh, p, i, rv);
        }
        if (!shifts_first) shift_updates_site<ST, R>(rin, P, stride, y, g.Vh, p, i, na, sidx, sw, sb, w0);
    }
    grid_reduce_warp<1>(v, rs, ShiftFinL{s});
}

// p_0 = r_{k+1} + beta_k p_0 (fused form; nw words)
template <typename ST>
__global__ void __launch_bounds__(kBlock) k_ms_p0(const MsState *s, const ST *__restrict__ rb0,
                                                  const ST *__restrict__ rb1, ST *__restrict__ P0, long nw) {
    if (s->done) return;
    const ST *__restrict__ r = (s->iter & 1) ? rb1 : rb0;
    using A = typename Word<ST>::A;
    constexpr int N = Word<ST>::N;
    const A b = A(s->beta_prev);
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (long)gridDim.x * blockDim.x) {
        A rv[N], pv[N];
        Word<ST>::get(r[k], rv);
        Word<ST>::get(P0[k], pv);
#pragma unroll
        for (int e = 0; e < N; e++) pv[e] = fma_r(b, pv[e], rv[e]);
        P0[k] = Word<ST>::put(pv);
    }
}

struct InitFin {
    MsState *s;
    __device__ void operator()(const double *v) const {
        s->bb = v[0];
        s->rr = v[0];
        s->pp = v[0];   // p_0 = b
        if (v[0] == 0.0) s->done = 1;
        if (!isfinite(v[0])) {
            s->status = 1;
            s->done = 1;
        }
    }
};

// r = y = p_l = b ; ||b||^2
template <typename ST>
__global__ void k_ms_init(MsState *s, const ST *__restrict__ b, ST *r, ST *y, ST *P, long stride, long nw,
                          int n, RedScratch rs) {
    constexpr int N = Word<ST>::N;
    using A = typename Word<ST>::A;
    A v[1] = {A(0)};
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (long)gridDim.x * blockDim.x) {
        const ST w = b[k];
        r[k] = w;
        y[k] = w;
        for (int l = 0; l < n; l++) P[l * stride + k] = w;
        A e[N], a = A(0);
        Word<ST>::get(w, e);
#pragma unroll
        for (int q = 0; q < N; q++) a += e[q] * e[q];
        v[0] += a;
    }
    grid_reduce<1>(v, rs, InitFin{s});
}

inline int stream_grid(long n) {
    long b = (n + kBlock - 1) / kBlock;
    const long cap = 152L * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

// ---- 16-bit shifted directions (one thread per site: the FP16 words share a norm)
// y += sum_l w_l a^l p_l ; p_l = zeta_l r + b^l p_l, with p_0 in FP32 and p_l (l >= 1)
// in FP16 with a per-site scale (BF = false) or in BF16 (BF = true); the last block
// retires finished shifts as k_ms_shifts does.
template <bool BF>
__device__ __forceinline__ void load_p16(const MsVectorsH &v, int l, int Vh, int p, int i, cpx<float> pv[12]) {
    if (BF) load_spinor<float>(Bf16SpinorC{v.ph + (size_t)(l - 1) * v.words_h}, Vh, p, i, pv);
    else load_spinor<float>(HalfSpinorC{v.ph + (size_t)(l - 1) * v.words_h, v.pn + (size_t)(l - 1) * 2 * Vh}, Vh, p,
                            i, pv);
}
template <bool BF>
__device__ __forceinline__ void store_p16(const MsVectorsH &v, int l, int Vh, int p, int i, const cpx<float> pv[12]) {
    if (BF) store_spinor<float>(Bf16Spinor{v.ph + (size_t)(l - 1) * v.words_h}, Vh, p, i, pv);
    else store_spinor<float>(HalfSpinor{v.ph + (size_t)(l - 1) * v.words_h, v.pn + (size_t)(l - 1) * 2 * Vh}, Vh, p,
                             i, pv);
}

template <bool BF>
__global__ void __launch_bounds__(kBlock) k_ms_shifts_half(Geom g, MsState *s, MsVectorsH v, unsigned *counter) {
    __shared__ float sw[kMaxPoles], sb[kMaxPoles];
    __shared__ int sidx[kMaxPoles];
    __shared__ int sact, sdone;
    if (threadIdx.x == 0) {
        sdone = s->done;
        int na = 0;
        if (sdone != 1)
            for (int l = 0; l < s->n; l++)
                if (s->active[l]) {
                    sidx[na] = l;
                    sw[na] = (float)(s->w[l] * s->alpha_l[l]);
                    sb[na] = (float)s->beta_l[l];
                    na++;
                }
        sact = na;
    }
    __syncthreads();
    if (sdone == 1) return;
    const int na = sact;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.V; k += gridDim.x * blockDim.x) {
        const int p = k >= g.Vh, i = k - p * g.Vh;   // no neighbours: plain parity-major order
        cpx<float> rv[12], yv[12], pv[12];
        load_spinor<float>(v.r, g.Vh, p, i, rv);
        load_spinor<float>(v.y, g.Vh, p, i, yv);
        for (int a = 0; a < na; a++) {
            const int l = sidx[a];
            const float wl = sw[a], bl = sb[a];
            if (l == 0) load_spinor<float>(v.p0, g.Vh, p, i, pv);
            else load_p16<BF>(v, l, g.Vh, p, i, pv);
#pragma unroll
            for (int c = 0; c < 12; c++) {
                yv[c] = yv[c] + wl * pv[c];
                pv[c] = rv[c] + bl * pv[c];
            }
            if (l == 0) store_spinor<float>(v.p0, g.Vh, p, i, pv);
            else store_p16<BF>(v, l, g.Vh, p, i, pv);
        }
        store_spinor<float>(v.y, g.Vh, p, i, yv);
    }
    if (grid_last_block(counter)) {
        for (int l = threadIdx.x; l < s->n; l += blockDim.x)
            if (s->active[l] == 2) s->active[l] = 0;
        __syncthreads();
        if (threadIdx.x == 0 && s->done == 2) s->done = 1;
    }
}

// r = y = p_0 = b in FP32, p_l = b in FP16 or BF16 (l >= 1) ; ||b||^2
template <bool BF>
__global__ void k_ms_init_half(Geom g, MsState *s, MsVectorsH v, const float4 *__restrict__ b, int n, RedScratch rs) {
    float acc[1] = {0.f};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.V; k += gridDim.x * blockDim.x) {
        const int p = k >= g.Vh, i = k - p * g.Vh;
        cpx<float> bv[12];
        load_spinor<float>(b, g.Vh, p, i, bv);
        store_spinor<float>(v.r, g.Vh, p, i, bv);
        store_spinor<float>(v.y, g.Vh, p, i, bv);
        store_spinor<float>(v.p0, g.Vh, p, i, bv);
        for (int l = 1; l < n; l++) store_p16<BF>(v, l, g.Vh, p, i, bv);
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < 12; c++) a += norm2(bv[c]);
        acc[0] += a;
    }
    grid_reduce<1>(acc, rs, InitFin{s});
}

template <typename R, typename LT, typename ST>
cudaError_t ms_iter_t(const Geom &g, const LT *U, R m0, MsState *s, MsVectors<ST> v, RedScratch rs,
                      cudaStream_t st, cudaEvent_t *ev, unsigned ev_flags) {
    const int tps = sizeof(R) == 8 ? g.tps64 : g.tps32;
    const int gs = red_grid(4L * g.V);
    const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<R>::value, kMaxRedBlocks);
    cudaError_t e;
    if (ev && (e = cudaEventRecordWithFlags(ev[0], st, ev_flags)) != cudaSuccess) return e;
    // the fused form pays where the stencil waits on memory (FP32); the FP64 and float-float
    // stencils are bound by arithmetic that the shift updates would add to
    if (tps == 4 || sizeof(R) != 4) {   // three-kernel form (4 or 1 threads per site)
        if (tps == 4) k_ms_q4<R, LT, ST><<<gs, kBlock, 0, st>>>(g, U, m0 + (R)4, s, v.p, v.t, rs);
        else k_ms_q<R, LT, ST, false><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + (R)4, s, v.p, v.t, rs, ls.spb);
        if (ev && (e = cudaEventRecordWithFlags(ev[1], st, ev_flags)) != cudaSuccess) return e;
        if (tps == 4) k_ms_r4<R, LT, ST><<<gs, kBlock, 0, st>>>(g, U, m0 + (R)4, s, v.t, v.p, v.r, rs);
        else k_ms_r<R, LT, ST><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + (R)4, s, v.t, v.p, v.r, rs, ls.spb);
        if (ev && (e = cudaEventRecordWithFlags(ev[2], st, ev_flags)) != cudaSuccess) return e;
        k_ms_shifts<ST><<<stream_grid(v.stride), kBlock, 0, st>>>(s, v.r, v.y, v.p, v.stride, v.stride, rs.counter);
    } else {          // fused form
        k_ms_q<R, LT, ST, true><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + (R)4, s, v.p, v.t, rs, ls.spb);
        if (ev && (e = cudaEventRecordWithFlags(ev[1], st, ev_flags)) != cudaSuccess) return e;
        k_ms_rf<R, LT, ST><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + (R)4, s, v.t, v.p, v.stride, v.r, v.r2, v.y,
                                                         rs, ls.spb);
        if (ev && (e = cudaEventRecordWithFlags(ev[2], st, ev_flags)) != cudaSuccess) return e;
        k_ms_p0<ST><<<stream_grid(v.stride), kBlock, 0, st>>>(s, v.r, v.r2, v.p, v.stride);
    }
    if (ev && (e = cudaEventRecordWithFlags(ev[3], st, ev_flags)) != cudaSuccess) return e;
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace

cudaError_t ms_init_f64(const Geom &g, int n, MsState *s, MsVectors<double2> v, const double2 *b, RedScratch rs,
                        cudaStream_t st) {
    k_ms_init<double2><<<red_grid(v.stride), kBlock, 0, st>>>(s, b, v.r, v.y, v.p, v.stride, v.stride, n, rs);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t ms_init_f32(const Geom &g, int n, MsState *s, MsVectors<float4> v, const float4 *b, RedScratch rs,
                        cudaStream_t st) {
    k_ms_init<float4><<<red_grid(v.stride), kBlock, 0, st>>>(s, b, v.r, v.y, v.p, v.stride, v.stride, n, rs);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t ms_iter_f64(const Geom &g, const double2 *U, double m0, MsState *s, MsVectors<double2> v,
                        RedScratch rs, cudaStream_t st, cudaEvent_t *ev, unsigned ev_flags) {
    return ms_iter_t<double, double2, double2>(g, U, m0, s, v, rs, st, ev, ev_flags);
}
cudaError_t ms_iter_f32(const Geom &g, const float4 *U, float m0, MsState *s, MsVectors<float4> v,
                        RedScratch rs, cudaStream_t st, cudaEvent_t *ev, unsigned ev_flags) {
    return ms_iter_t<float, float4, float4>(g, U, m0, s, v, rs, st, ev, ev_flags);
}

// float-float multishift: the same three kernels on float-float vectors and links (one
// thread per site); the scalar recurrences stay FP64 on the device.
cudaError_t ms_init_ff(const Geom &g, int n, MsState *s, MsVectors<ffw> v, const ffw *b, RedScratch rs,
                       cudaStream_t st) {
    k_ms_init<ffw><<<red_grid(v.stride), kBlock, 0, st>>>(s, b, v.r, v.y, v.p, v.stride, v.stride, n, rs);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t ms_iter_ff(const Geom &g, const ffw *U, double m0, MsState *s, MsVectors<ffw> v, RedScratch rs,
                       cudaStream_t st, cudaEvent_t *ev, unsigned ev_flags) {
    const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<ff>::value, kMaxRedBlocks);
    const ff m4(m0 + 4.0);
    cudaError_t e;
    if (ev && (e = cudaEventRecordWithFlags(ev[0], st, ev_flags)) != cudaSuccess) return e;
    k_ms_q<ff, ffw, ffw, false><<<ls.grid, ls.block, 0, st>>>(g, U, m4, s, v.p, v.t, rs, ls.spb);
    if (ev && (e = cudaEventRecordWithFlags(ev[1], st, ev_flags)) != cudaSuccess) return e;
    k_ms_r<ff, ffw, ffw><<<ls.grid, ls.block, 0, st>>>(g, U, m4, s, v.t, v.p, v.r, rs, ls.spb);
    if (ev && (e = cudaEventRecordWithFlags(ev[2], st, ev_flags)) != cudaSuccess) return e;
    k_ms_shifts<ffw><<<stream_grid(v.stride), kBlock, 0, st>>>(s, v.r, v.y, v.p, v.stride, v.stride, rs.counter);
    if (ev && (e = cudaEventRecordWithFlags(ev[3], st, ev_flags)) != cudaSuccess) return e;
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace ovl

namespace ovl {
cudaError_t ms_init_half(const Geom &g, int n, MsState *s, MsVectorsH v, const float4 *b, RedScratch rs, bool bf16,
                         cudaStream_t st) {
    if (bf16) k_ms_init_half<true><<<red_grid(g.V), kBlock, 0, st>>>(g, s, v, b, n, rs);
    else k_ms_init_half<false><<<red_grid(g.V), kBlock, 0, st>>>(g, s, v, b, n, rs);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t ms_iter_half(const Geom &g, const float4 *U, float m0, MsState *s, MsVectorsH v, RedScratch rs, bool bf16,
                         cudaStream_t st, cudaEvent_t *ev, unsigned ev_flags) {
    const LaunchShape ls = balanced_shape(g.V, g.nsm, MinBlocks<float>::value, kMaxRedBlocks);
    cudaError_t e;
    if (ev && (e = cudaEventRecordWithFlags(ev[0], st, ev_flags)) != cudaSuccess) return e;
    k_ms_q<float, float4, float4, false><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + 4.f, s, v.p0, v.t, rs, ls.spb);
    if (ev && (e = cudaEventRecordWithFlags(ev[1], st, ev_flags)) != cudaSuccess) return e;
    k_ms_r<float, float4, float4><<<ls.grid, ls.block, 0, st>>>(g, U, m0 + 4.f, s, v.t, v.p0, v.r, rs, ls.spb);
    if (ev && (e = cudaEventRecordWithFlags(ev[2], st, ev_flags)) != cudaSuccess) return e;
    const int gsh = balanced_shape(g.V, g.nsm, 2, 1 << 30).grid;
    if (bf16) k_ms_shifts_half<true><<<gsh, kBlock, 0, st>>>(g, s, v, rs.counter);
    else k_ms_shifts_half<false><<<gsh, kBlock, 0, st>>>(g, s, v, rs.counter);
    if (ev && (e = cudaEventRecordWithFlags(ev[3], st, ev_flags)) != cudaSuccess) return e;
    count_launches(3);
    return cudaGetLastError();
}
}  // namespace ovl

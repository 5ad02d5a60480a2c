// Several right-hand sides at once: the multi-RHS Wilson stencil and the batched
// multishift CG that runs one independent Zolotarev sign evaluation per right-hand side
// in lock-step.
//
// The FP32 multi-RHS stencil has three kernels, chosen per lattice shape by the autotuner
// (Geom::mrhs32): the right-hand sides in pairs looped inside each site's thread
// (k_wilson_mrhs_pairs), blocks of 32 sites x one warp per right-hand side (k_wilson_mrhs), or
// the links staged in shared memory with the right-hand sides looped (k_wilson_mrhs_links).
// The FP64 stencil and the batched multishift kernels use thread blocks of 32 sites x nr
// right-hand sides (threadIdx.x = site, threadIdx.y = right-hand side). The nr threads of one site need the same eight links; running them
// in one block makes the repeats hit L1, so DRAM sees each link once per block of
// right-hand sides: per site and right-hand side the stencil moves 48 / nr link reals
// plus 48 spinor reals instead of 96. Each warp holds one right-hand side, so warp sums
// are per-right-hand-side partial sums and the per-shift scalar update (ShiftFin) runs
// in the warp of its right-hand side.
#include "internal.h"
#include "reduce.cuh"
#include "wilson_site.cuh"

namespace ovl {

namespace {

constexpr int kTile = 32;   // sites per block (one warp per right-hand side)

__device__ __forceinline__ int tile_site(int bx) { return bx * kTile + (int)threadIdx.x; }

template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(384) k_wilson_mrhs(Geom g, const LT *__restrict__ U, const ST *__restrict__ in,
                                                     ST *__restrict__ out, long stride, int nrhs, R m4, int g5, R a,
                                                     const ST *z, R b) {
    const int rhs = blockIdx.y * blockDim.y + threadIdx.y;
    const int t = tile_site(blockIdx.x);
    if (rhs >= nrhs || t >= g.V) return;
    int p, i;
    site_of_thread(t, p, i);
    const ST *x = in + rhs * stride;
    cpx<R> hop[12], own[12], res[12];
    wilson_hop<R>(g, U, x, p, i, hop);
    load_spinor<R>(x, g.Vh, p, i, own);
    wilson_combine<R>(m4, own, hop, res);
    if (g5) apply_g5(res);
    if (z) {
        cpx<R> zz[12];
        load_spinor<R>(z + rhs * stride, g.Vh, p, i, zz);
#pragma unroll
        for (int c = 0; c < 12; c++) res[c] = a * res[c] + b * zz[c];
    } else {
#pragma unroll
        for (int c = 0; c < 12; c++) res[c] = a * res[c];
    }
    store_spinor<R>(out + rhs * stride, g.Vh, p, i, res);
}

// FP32 multi-RHS stencil: each thread owns one site in the single-RHS order (blocks of up to 256
// consecutive sites, both parities interleaved, so most x3 and x2 neighbours of a block hit L1)
// and loops over the right-hand sides two at a time, applying every link it loads to both
// (wilson_hop2). A block of 32 sites x nr right-hand sides (k_wilson_mrhs) shares the links
// across right-hand sides too, but its blocks span one x3 row, so the x2 neighbours miss L1 and
// the spinor gathers that bound this stencil grow; measured per right-hand side at 12 of them it
// ran 1.16x the single-RHS time at 64x32^3, this loop 0.95x (32^4: 0.88x, 16^4: 0.52x).
__global__ void __launch_bounds__(kBlock, 2) k_wilson_mrhs_pairs(Geom g, const float4 *__restrict__ U,
                                                               const float4 *__restrict__ in, float4 *__restrict__ out,
                                                               long stride, int nrhs, float m4, int g5, float a,
                                                               const float4 *z, float b, int spb) {
    const int t = blockIdx.x * spb + threadIdx.x;
    if (threadIdx.x >= spb || t >= g.V) return;
    int p, i;
    site_of_thread(t, p, i);
#pragma unroll 1
    for (int r = 0; r < nrhs; r += 2) {
        const bool two = r + 1 < nrhs;
        const float4 *x0 = in + r * stride, *x1 = two ? x0 + stride : x0;
        cpx<float> hop[2][12];
        wilson_hop2<float>(g, U, x0, x1, p, i, hop[0], hop[1]);
#pragma unroll
        for (int f = 0; f < 2; f++) {
            if (f == 1 && !two) break;
            const int rhs = r + f;
            cpx<float> own[12], res[12];
            load_spinor<float>(in + rhs * stride, g.Vh, p, i, own);
            wilson_combine<float>(m4, own, hop[f], res);
            if (g5) apply_g5(res);
            if (z) {
                cpx<float> zz[12];
                load_spinor<float>(z + rhs * stride, g.Vh, p, i, zz);
#pragma unroll
                for (int c = 0; c < 12; c++) res[c] = a * res[c] + b * zz[c];
            } else {
#pragma unroll
                for (int c = 0; c < 12; c++) res[c] = a * res[c];
            }
            store_spinor<float>(out + rhs * stride, g.Vh, p, i, res);
        }
    }
}

// FP32 multi-RHS stencil with the links staged per thread: each thread owns one site in the
// single-RHS order, copies its eight links (4 forward at the site, 4 backward at the neighbours,
// rows 0-1: 24 words) and its eight neighbour indices into its own column of shared memory once,
// and applies them to every right-hand side in turn, so the links leave L2 once per launch
// instead of once per right-hand side. The shared memory (about 100 KB per 256-thread block)
// comes out of L1, which the neighbour spinors would otherwise hit in: measured at 12
// right-hand sides it is the best of the three kernels at 16^4 and the worst at 32^4 and above,
// which is why the autotuner chooses per lattice shape.
constexpr int kLinkSlotWords = 24;

template <int MU>
__device__ __forceinline__ void hop_dir_slot(const Geom &g, const float4 *__restrict__ in, int q, const int *nb,
                                             int x0, const float4 *sl, int S, cpx<float> acc[12]) {
    const int jf = nb[MU * S], jb = nb[(4 + MU) * S];
    {   // forward: link words MU*3 .. MU*3+2
        cpx<float> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<float>(in, g.Vh, q, jf, s);
        proj_fwd(MU, s, h0, h1);
        if (MU == 0) flip_half(h0, h1, g.antiperiodic && x0 == g.L[0] - 1);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 v = sl[(MU * 3 + c) * S];
            u[(2 * c) / 3][(2 * c) % 3] = cpx<float>{v.x, v.y};
            u[(2 * c + 1) / 3][(2 * c + 1) % 3] = cpx<float>{v.z, v.w};
        }
        reconstruct_row2(u);
        su3_mul(u, h0, a0);
        su3_mul(u, h1, a1);
        acc_fwd<MU == 0>(MU, acc, a0, a1);
    }
    {   // backward: link words 12 + MU*3 ..
        cpx<float> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
        load_spinor<float>(in, g.Vh, q, jb, s);
        proj_bwd(MU, s, h0, h1);
        if (MU == 0) flip_half(h0, h1, g.antiperiodic && x0 == 0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 v = sl[(12 + MU * 3 + c) * S];
            u[(2 * c) / 3][(2 * c) % 3] = cpx<float>{v.x, v.y};
            u[(2 * c + 1) / 3][(2 * c + 1) % 3] = cpx<float>{v.z, v.w};
        }
        reconstruct_row2(u);
        su3_dag_mul(u, h0, a0);
        su3_dag_mul(u, h1, a1);
        acc_bwd(MU, acc, a0, a1);
    }
}

__global__ void __launch_bounds__(kBlock, 2) k_wilson_mrhs_links(Geom g, const float4 *__restrict__ U,
                                                               const float4 *__restrict__ in, float4 *__restrict__ out,
                                                               long stride, int nrhs, float m4, int g5, float a,
                                                               const float4 *z, float b, int spb) {
    // [kLinkSlotWords][blockDim.x] links, then [8][blockDim.x] neighbour indices (forward, backward)
    extern __shared__ float4 link_slots[];
    const int t = blockIdx.x * spb + threadIdx.x;
    if (threadIdx.x >= spb || t >= g.V) return;
    int p, i;
    site_of_thread(t, p, i);
    int x[4];
    eo_coords(g, p, i, x);
    const int q = 1 - p, S = blockDim.x;
    float4 *sl = link_slots + threadIdx.x;
    int *nb = reinterpret_cast<int *>(link_slots + kLinkSlotWords * S) + threadIdx.x;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        int y[4] = {x[0], x[1], x[2], x[3]};
        y[mu] = x[mu] + 1 == g.L[mu] ? 0 : x[mu] + 1;
        nb[mu * S] = eo_index(g, y);
        y[mu] = x[mu] == 0 ? g.L[mu] - 1 : x[mu] - 1;
        const int jb = eo_index(g, y);
        nb[(4 + mu) * S] = jb;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            sl[(mu * 3 + c) * S] = __ldg(U + ((size_t)(p * 4 + mu) * 3 + c) * g.Vh + i);
            sl[(12 + mu * 3 + c) * S] = __ldg(U + ((size_t)(q * 4 + mu) * 3 + c) * g.Vh + jb);
        }
    }
    const int x0 = x[0];
    // each thread reads back only its own column: no barrier needed
#pragma unroll 1
    for (int r = 0; r < nrhs; r++) {
        const float4 *xin = in + r * stride;
        cpx<float> acc[12], own[12], res[12];
        hop_dir_slot<0>(g, xin, q, nb, x0, sl, S, acc);
        hop_dir_slot<1>(g, xin, q, nb, x0, sl, S, acc);
        hop_dir_slot<2>(g, xin, q, nb, x0, sl, S, acc);
        hop_dir_slot<3>(g, xin, q, nb, x0, sl, S, acc);
        load_spinor<float>(xin, g.Vh, p, i, own);
        wilson_combine<float>(m4, own, acc, res);
        if (g5) apply_g5(res);
        if (z) {
            cpx<float> zz[12];
            load_spinor<float>(z + r * stride, g.Vh, p, i, zz);
#pragma unroll
            for (int c = 0; c < 12; c++) res[c] = a * res[c] + b * zz[c];
        } else {
#pragma unroll
            for (int c = 0; c < 12; c++) res[c] = a * res[c];
        }
        store_spinor<float>(out + r * stride, g.Vh, p, i, res);
    }
}

// Per-right-hand-side grid reduction: warp y of every block holds the partial sums of
// right-hand side y (in T: FP32 kernels sum their warps in FP32); the last block sums each
// row in block order in FP64 and warp y runs fin(rhs, total, lane).
// partials: [nrhs][NV][kMaxRedBlocks].
template <int NV, typename T, typename Fin>
__device__ __forceinline__ void grid_reduce_rows(const T vt[NV], RedScratch rs, int nrhs, Fin fin) {
    __shared__ int is_last;
    const int y = threadIdx.y, lane = threadIdx.x;
    T v[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        v[k] = vt[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0 && y < nrhs)
#pragma unroll
        for (int k = 0; k < NV; k++)
            rs.partials[((size_t)y * NV + k) * kMaxRedBlocks + blockIdx.x] = (double)v[k];
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        unsigned t = atomicAdd(rs.counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (y < nrhs) {
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            s[k] = 0.0;
            for (int bb = lane; bb < (int)gridDim.x; bb += 32)
                s[k] += __ldcg(rs.partials + ((size_t)y * NV + k) * kMaxRedBlocks + bb);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], off);
            s[k] = __shfl_sync(0xffffffffu, s[k], 0);
        }
        fin(y, s, lane);
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) *rs.counter = 0u;
}

struct AlphaFinB {
    MsState *st;
    __device__ void operator()(int y, const double *v, int lane) const {
        MsState *s = st + y;
        if (lane != 0 || s->done) return;
        const double pAp = v[0] + s->sigma[0] * v[1];
        const double a = s->rr / pAp;
        if (!(pAp > 0.0) || !isfinite(a)) {
            s->status = 1;
            s->done = 1;
            return;
        }
        s->alpha = a;
    }
};

// Shift scalars of right-hand side y (one warp, lane j handles shifts j, j + 32).
struct ShiftFinB {
    MsState *st;
    __device__ void operator()(int y, const double *v, int lane) const {
        MsState *s = st + y;
        if (s->done) return;   // uniform over the warp
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
        const double rnorm = sqrt(rr_new), tolb = s->tol * sqrt(s->bb);
        int any = 0;
        for (int l = lane; l < n; l += 32) {
            if (!s->active[l]) {
                s->alpha_l[l] = 0.0;
                continue;
            }
            double zn;
            if (l == 0) {
                zn = 1.0;
            } else {
                const double zz = s->zeta[l], zp = s->zeta_prev[l];
                const double den = a * bp * (zp - zz) + zp * ap * (1.0 + (s->sigma[l] - s->sigma[0]) * a);
                zn = (den != 0.0) ? zz * zp * ap / den : 0.0;
            }
            const double ratio = (s->zeta[l] != 0.0) ? zn / s->zeta[l] : 0.0;
            // directions stored as p~_l = p_l / zeta_l (see the header): y += w_l a zeta_new p~_l,
            // p~_l = r + b ratio p~_l
            s->alpha_l[l] = a * zn;
            s->beta_l[l] = beta * ratio;
            s->zeta_prev[l] = s->zeta[l];
            s->zeta[l] = zn;
            if (s->crit[l] * fabs(zn) * rnorm <= tolb) s->active[l] = 2;
            else any = 1;
        }
        any = __any_sync(0xffffffffu, any);
        __syncwarp();
        if (lane == 0) {
            if (any && s->active[0] == 2) s->active[0] = 1;
            s->alpha_prev = a;
            s->beta_prev = beta;
            s->rr = rr_new;
            s->iter += 1;
            if (!any) s->done = 2;
        }
    }
};

// t_y = gamma5 D_W p0_y ; per y: ||t_y||^2, ||p0_y||^2 -> alpha_y
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(384) k_msb_q(Geom g, const LT *__restrict__ U, R m4, MsState *st, int nrhs,
                                               const ST *__restrict__ p0, long pstride, ST *__restrict__ t,
                                               long stride, RedScratch rs) {
    const int y = threadIdx.y;
    const bool live = y < nrhs && !st[y].done;
    R v[2] = {0, 0};
    if (live) {
        const ST *x = p0 + y * pstride;
        for (int k = tile_site(blockIdx.x); k < g.V; k += gridDim.x * kTile) {
            int p, i;
            site_of_thread(k, p, i);
            cpx<R> hop[12], own[12], res[12];
            wilson_hop<R>(g, U, x, p, i, hop);
            load_spinor<R>(x, g.Vh, p, i, own);
            wilson_combine<R>(m4, own, hop, res);
            apply_g5(res);
            store_spinor<R>(t + y * stride, g.Vh, p, i, res);
            R a0 = 0, a1 = 0;
#pragma unroll
            for (int c = 0; c < 12; c++) {
                a0 += norm2(res[c]);
                a1 += norm2(own[c]);
            }
            v[0] += a0;
            v[1] += a1;
        }
    }
    grid_reduce_rows<2>(v, rs, nrhs, AlphaFinB{st});
}

// r_y -= alpha_y (gamma5 D_W t_y + sigma0_y p0_y) ; ||r_y||^2 -> shift scalars of y
template <typename R, typename LT, typename ST>
__global__ void __launch_bounds__(384) k_msb_r(Geom g, const LT *__restrict__ U, R m4, MsState *st, int nrhs,
                                               const ST *__restrict__ t, const ST *__restrict__ p0, long pstride,
                                               ST *__restrict__ r, long stride, RedScratch rs) {
    const int y = threadIdx.y;
    const bool live = y < nrhs && !st[y].done;
    R v[1] = {0};
    if (live) {
        const R alpha = (R)st[y].alpha, sig0 = (R)st[y].sigma[0];
        const ST *tt = t + y * stride, *pp = p0 + y * pstride;
        ST *rr = r + y * stride;
        for (int k = tile_site(blockIdx.x); k < g.V; k += gridDim.x * kTile) {
            int p, i;
            site_of_thread(k, p, i);
            cpx<R> hop[12], own[12], res[12], pv[12], rv[12];
            wilson_hop<R>(g, U, tt, p, i, hop);
            load_spinor<R>(tt, g.Vh, p, i, own);
            wilson_combine<R>(m4, own, hop, res);
            apply_g5(res);
            load_spinor<R>(pp, g.Vh, p, i, pv);
            load_spinor<R>(rr, g.Vh, p, i, rv);
            R a0 = 0;
#pragma unroll
            for (int c = 0; c < 12; c++) {
                rv[c] = rv[c] - alpha * (res[c] + sig0 * pv[c]);
                a0 += norm2(rv[c]);
            }
            v[0] += a0;
            store_spinor<R>(rr, g.Vh, p, i, rv);
        }
    }
    grid_reduce_rows<1>(v, rs, nrhs, ShiftFinB{st});
}

template <typename ST> struct WordB;
template <> struct WordB<double2> {
    static constexpr int N = 2;
    using A = double;
    __device__ static void get(const double2 &w, A *o) { o[0] = w.x; o[1] = w.y; }
    __device__ static double2 put(const A *o) { return make_double2(o[0], o[1]); }
};
template <> struct WordB<float4> {
    static constexpr int N = 4;
    using A = float;
    __device__ static void get(const float4 &w, A *o) { o[0] = w.x; o[1] = w.y; o[2] = w.z; o[3] = w.w; }
    __device__ static float4 put(const A *o) { return make_float4(o[0], o[1], o[2], o[3]); }
};

// Shift updates of right-hand side blockIdx.y (words of ST). P holds, per right-hand
// side, n directions of `stride` words: P + (y * n + l) * stride.
template <typename ST>
__global__ void __launch_bounds__(kBlock) k_msb_shifts(MsState *st, int npole, const ST *__restrict__ r,
                                                       ST *__restrict__ yv_, ST *__restrict__ P, long stride,
                                                       unsigned *counters) {
    using A = typename WordB<ST>::A;
    constexpr int N = WordB<ST>::N;
    __shared__ A sw[kMaxPoles], sb[kMaxPoles];
    __shared__ int sidx[kMaxPoles];
    __shared__ int sact, sdone;
    const int y = blockIdx.y;
    MsState *s = st + y;
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
    if (sdone == 1) return;   // uniform over the blocks of this right-hand side
    const int na = sact;
    const ST *ry = r + y * stride;
    ST *yy = yv_ + y * stride;
    ST *Py = P + (long)y * npole * stride;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < stride; k += (long)gridDim.x * blockDim.x) {
        A rv[N], yv[N];
        WordB<ST>::get(ry[k], rv);
        WordB<ST>::get(yy[k], yv);
        for (int a0 = 0; a0 < na; a0 += 4) {
            ST w[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (a0 + u < na) w[u] = Py[(long)sidx[a0 + u] * stride + k];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (a0 + u >= na) break;
                A pv[N];
                WordB<ST>::get(w[u], pv);
                const A wl = sw[a0 + u], bl = sb[a0 + u];
#pragma unroll
                for (int e = 0; e < N; e++) {
                    yv[e] += wl * pv[e];
                    pv[e] = rv[e] + bl * pv[e];
                }
                Py[(long)sidx[a0 + u] * stride + k] = WordB<ST>::put(pv);
            }
        }
        yy[k] = WordB<ST>::put(yv);
    }
    if (grid_last_block(counters + y)) {   // last block of this right-hand side's row
        for (int l = threadIdx.x; l < s->n; l += blockDim.x)
            if (s->active[l] == 2) s->active[l] = 0;
        __syncthreads();
        if (threadIdx.x == 0 && s->done == 2) s->done = 1;
    }
}

struct InitFinB {
    MsState *st;
    __device__ void operator()(int y, const double *v, int lane) const {
        if (lane != 0) return;
        MsState *s = st + y;
        s->bb = v[0];
        s->rr = v[0];
        if (v[0] == 0.0) s->done = 1;
        if (!isfinite(v[0])) {
            s->status = 1;
            s->done = 1;
        }
    }
};

// r_y = y_y = p_{y,l} = b_y ; ||b_y||^2   (32 x nrhs blocks over storage words)
template <typename ST>
__global__ void __launch_bounds__(384) k_msb_init(MsState *st, int nrhs, int npole, const ST *__restrict__ b, ST *r,
                                                  ST *yv_, ST *P, long stride, RedScratch rs) {
    using A = typename WordB<ST>::A;
    constexpr int N = WordB<ST>::N;
    const int y = threadIdx.y;
    A v[1] = {0};
    if (y < nrhs) {
        for (long k = (long)blockIdx.x * kTile + threadIdx.x; k < stride; k += (long)gridDim.x * kTile) {
            const ST w = b[y * stride + k];
            r[y * stride + k] = w;
            yv_[y * stride + k] = w;
            for (int l = 0; l < npole; l++) P[((long)y * npole + l) * stride + k] = w;
            A e[N], a = 0;
            WordB<ST>::get(w, e);
#pragma unroll
            for (int q = 0; q < N; q++) a += e[q] * e[q];
            v[0] += a;
        }
    }
    grid_reduce_rows<1>(v, rs, nrhs, InitFinB{st});
}

inline int tiles_grid(long n_items) {
    long b = (n_items + kTile - 1) / kTile;
    if (b > kMaxRedBlocks) b = kMaxRedBlocks;
    return (int)(b < 1 ? 1 : b);
}

inline int stream_grid_b(long n) {
    long b = (n + kBlock - 1) / kBlock;
    const long cap = (long)device_sm_count() * 4;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// out_y = a [gamma5] D_W(m0) in_y + b z_y, y < nrhs (nrhs <= 12), vectors `stride` words apart
cudaError_t wilson_batch_f64(const Geom &g, const double2 *U, const double2 *in, double2 *out, long stride, int nrhs,
                             double m0, int g5, double a, const double2 *z, double b, cudaStream_t st) {
    k_wilson_mrhs<double, double2, double2><<<dim3((g.V + kTile - 1) / kTile, 1), dim3(kTile, nrhs), 0, st>>>(
        g, U, in, out, stride, nrhs, m0 + 4.0, g5, a, z, b);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t wilson_batch_f32(const Geom &g, const float4 *U, const float4 *in, float4 *out, long stride, int nrhs,
                             float m0, int g5, float a, const float4 *z, float b, cudaStream_t st) {
    const int kern = nrhs > 6 ? g.mrhs32l : g.mrhs32;
    if (nrhs > 1 && kern == 3) {
        static unsigned attr_set = 0;   // devices whose dynamic shared memory limit is raised
        int dev = 0;
        const int most = kBlock * (kLinkSlotWords * (int)sizeof(float4) + 8 * (int)sizeof(int));
        if (cudaGetDevice(&dev) == cudaSuccess && dev < 32 && !(attr_set & (1u << dev))) {
            const cudaError_t e = cudaFuncSetAttribute(k_wilson_mrhs_links, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       most);
            if (e != cudaSuccess) return e;
            attr_set |= 1u << dev;
        }
        const LaunchShape ls = balanced_shape(g.V, g.nsm, 2, 1 << 30);
        const size_t smem = (size_t)ls.block * (kLinkSlotWords * sizeof(float4) + 8 * sizeof(int));
        k_wilson_mrhs_links<<<ls.grid, ls.block, smem, st>>>(g, U, in, out, stride, nrhs, m0 + 4.f, g5, a, z, b,
                                                             ls.spb);
    } else if (nrhs > 1 && kern != 2) {
        const LaunchShape ls = balanced_shape(g.V, g.nsm, 2, 1 << 30);
        k_wilson_mrhs_pairs<<<ls.grid, ls.block, 0, st>>>(g, U, in, out, stride, nrhs, m0 + 4.f, g5, a, z, b,
                                                          ls.spb);
    } else
        k_wilson_mrhs<float, float4, float4><<<dim3((g.V + kTile - 1) / kTile, 1), dim3(kTile, nrhs), 0, st>>>(
            g, U, in, out, stride, nrhs, m0 + 4.f, g5, a, z, b);
    count_launches(1);
    return cudaGetLastError();
}

template <typename ST>
static cudaError_t msb_init_t(const Geom &g, int nrhs, int npole, MsState *st, MsBatch<ST> v, const ST *b,
                              RedScratch rs, cudaStream_t s) {
    k_msb_init<ST><<<tiles_grid(v.stride), dim3(kTile, nrhs), 0, s>>>(st, nrhs, npole, b, v.r, v.y, v.p, v.stride, rs);
    count_launches(1);
    return cudaGetLastError();
}

template <typename R, typename LT, typename ST>
static cudaError_t msb_iter_t(const Geom &g, const LT *U, R m0, int nrhs, int npole, MsState *st, MsBatch<ST> v,
                              RedScratch rs, unsigned *counters, cudaStream_t s) {
    const int gx = tiles_grid(g.V);
    // p_0 of right-hand side y is direction 0 of its block: P + y * npole * stride
    k_msb_q<R, LT, ST><<<gx, dim3(kTile, nrhs), 0, s>>>(g, U, m0 + (R)4, st, nrhs, v.p, (long)npole * v.stride, v.t,
                                                          v.stride, rs);
    k_msb_r<R, LT, ST><<<gx, dim3(kTile, nrhs), 0, s>>>(g, U, m0 + (R)4, st, nrhs, v.t, v.p, (long)npole * v.stride,
                                                          v.r, v.stride, rs);
    k_msb_shifts<ST><<<dim3(stream_grid_b(v.stride), nrhs), kBlock, 0, s>>>(st, npole, v.r, v.y, v.p, v.stride,
                                                                             counters);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t msb_init_f64(const Geom &g, int nrhs, int npole, MsState *st, MsBatch<double2> v, const double2 *b,
                         RedScratch rs, cudaStream_t s) {
    return msb_init_t<double2>(g, nrhs, npole, st, v, b, rs, s);
}
cudaError_t msb_init_f32(const Geom &g, int nrhs, int npole, MsState *st, MsBatch<float4> v, const float4 *b,
                         RedScratch rs, cudaStream_t s) {
    return msb_init_t<float4>(g, nrhs, npole, st, v, b, rs, s);
}
cudaError_t msb_iter_f64(const Geom &g, const double2 *U, double m0, int nrhs, int npole, MsState *st,
                         MsBatch<double2> v, RedScratch rs, unsigned *counters, cudaStream_t s) {
    return msb_iter_t<double, double2, double2>(g, U, m0, nrhs, npole, st, v, rs, counters, s);
}
cudaError_t msb_iter_f32(const Geom &g, const float4 *U, float m0, int nrhs, int npole, MsState *st,
                         MsBatch<float4> v, RedScratch rs, unsigned *counters, cudaStream_t s) {
    return msb_iter_t<float, float4, float4>(g, U, m0, nrhs, npole, st, v, rs, counters, s);
}

}  // namespace ovl

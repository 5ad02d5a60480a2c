// Schwarz alternating procedure (SAP) for the Wilson-Dirac operator D_W(m0):
// the smoother of the inexact Wilson preconditioner.
//
// The paper preconditions with D_W(m0_prec)^{-1} applied inexactly (Sec. 5.1) by
// DD-alpha-AMG, whose smoother is a red-black multiplicative Schwarz method. Here the
// Schwarz method itself preconditions a short flexible GMRES on D_W(m0_prec):
//
//   blocks: the lattice is cut into blocks of b0 x b1 x b2 x b3 sites, coloured by the
//           parity of the block coordinates (red-black over blocks);
//   one cycle, x <- x + sum over colour c of the block corrections:
//       r = v - D_W x                       (full-lattice stencil)
//       for every block B of colour c: solve D_BB e_B = r_B approximately,
//       x_B += e_B
//   where D_BB is D_W restricted to the block (hops leaving the block dropped).
//
// Block solve: a fixed number of minimal-residual steps, one CTA per block with one
// thread per block site, the block's residual and links held in shared memory:
//   e = 0, s = r_B;  repeat:  q = D_BB s,  alpha = <q, s>/<q, q>,  e += alpha s,  s -= alpha q.
#include "internal.h"
#include "reduce.cuh"
#include "sap.h"
#include "wilson_site.cuh"

namespace ovl {

namespace {

// Resident CTAs per SM the block kernel is compiled for: FP32 blocks (74 KB of shared
// memory for 4^4 sites) fit two per SM at 128 registers; FP64 blocks (196 KB) fit one.
template <typename R> struct SapMinBlocks { static constexpr int value = 2; };
template <> struct SapMinBlocks<double> { static constexpr int value = 1; };

// Shared-memory copies of a block's spinor and forward links in the word layouts of
// global memory, one 16-byte load per word: FP32 spinor float4 [6][nb] and links float4
// [4][3][nb] (rows 0 and 1, row 2 rebuilt in registers), FP64 spinor double2 [12][nb]
// and links double2 [4][9][nb]. Consecutive threads read consecutive words (no bank
// conflicts).
template <typename W> struct SapWords;
template <> struct SapWords<float4> { static constexpr int spinor = 6, link = 3; };
template <> struct SapWords<double2> { static constexpr int spinor = 12, link = 9; };

__device__ __forceinline__ void sm_load_sp(const float4 *s, int nb, int t, cpx<float> v[12]) {
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const float4 w = s[c * nb + t];
        v[2 * c] = cpx<float>{w.x, w.y};
        v[2 * c + 1] = cpx<float>{w.z, w.w};
    }
}
__device__ __forceinline__ void sm_load_sp(const double2 *s, int nb, int t, cpx<double> v[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) {
        const double2 w = s[c * nb + t];
        v[c] = cpx<double>{w.x, w.y};
    }
}
__device__ __forceinline__ void sm_store_sp(float4 *s, int nb, int t, const cpx<float> v[12]) {
#pragma unroll
    for (int c = 0; c < 6; c++) s[c * nb + t] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
}
__device__ __forceinline__ void sm_store_sp(double2 *s, int nb, int t, const cpx<double> v[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) s[c * nb + t] = make_double2(v[c].re, v[c].im);
}
__device__ __forceinline__ void sm_load_link(const float4 *u, int nb, int mu, int t, cpx<float> m[3][3]) {
    const float4 *b = u + mu * 3 * nb + t;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float4 w = b[c * nb];
        m[(2 * c) / 3][(2 * c) % 3] = cpx<float>{w.x, w.y};
        m[(2 * c + 1) / 3][(2 * c + 1) % 3] = cpx<float>{w.z, w.w};
    }
    reconstruct_row2(m);
}
__device__ __forceinline__ void sm_load_link(const double2 *u, int nb, int mu, int t, cpx<double> m[3][3]) {
    const double2 *b = u + mu * 9 * nb + t;
#pragma unroll
    for (int c = 0; c < 9; c++) {
        const double2 w = b[c * nb];
        m[c / 3][c % 3] = cpx<double>{w.x, w.y};
    }
}
// The link words of U_mu at (p, i) in global memory, copied to block site t.
template <typename LT>
__device__ __forceinline__ void sm_copy_link(LT *u, int nb, int mu, int t, const LT *__restrict__ U, int Vh, int p,
                                             int i) {
    constexpr int W = SapWords<LT>::link;
    const LT *gw = U + ((size_t)(p * 4 + mu) * W) * Vh + i;
#pragma unroll
    for (int c = 0; c < W; c++) u[(mu * W + c) * nb + t] = __ldg(gw + (size_t)c * Vh);
}

// q = D_BB s at local site t (local coords l, extents bx), links of the block in smem.
template <typename R, typename LT, typename ST>
__device__ __forceinline__ void block_apply(const ST *s, const LT *u, int nb, int t, const int l[4], const int bx[4],
                                            const int stride[4], R m4, cpx<R> q[12]) {
    cpx<R> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cpx<R>{0, 0};
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        if (l[mu] + 1 < bx[mu]) {
            cpx<R> v[12], h0[3], h1[3], a0[3], a1[3], m[3][3];
            sm_load_sp(s, nb, t + stride[mu], v);
            sm_load_link(u, nb, mu, t, m);
            proj_fwd(mu, v, h0, h1);
            su3_mul(m, h0, a0);
            su3_mul(m, h1, a1);
            acc_fwd<false>(mu, acc, a0, a1);
        }
        if (l[mu] > 0) {
            cpx<R> v[12], h0[3], h1[3], a0[3], a1[3], m[3][3];
            sm_load_sp(s, nb, t - stride[mu], v);
            sm_load_link(u, nb, mu, t - stride[mu], m);
            proj_bwd(mu, v, h0, h1);
            su3_dag_mul(m, h0, a0);
            su3_dag_mul(m, h1, a1);
            acc_bwd(mu, acc, a0, a1);
        }
    }
    cpx<R> own[12];
    sm_load_sp(s, nb, t, own);
    wilson_combine<R>(m4, own, acc, q);
}

// MR step of a block solve: the block sums of Re<q, s>, Im<q, s> and |q|^2 (per warp by
// shuffles, then over warps in a fixed order by thread 0, all in R) and alpha = <q, s>/|q|^2,
// computed once by thread 0 and broadcast. Returns false when |q|^2 is not positive
// (uniform over the CTA). Every thread of the CTA must call it.
template <typename R>
__device__ __forceinline__ bool mr_alpha(R a0, R a1, R a2, cpx<R> &alpha) {
    __shared__ R red[3][32];
    __shared__ R bc[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, off);
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
        a2 += __shfl_down_sync(0xffffffffu, a2, off);
    }
    if (lane == 0) {
        red[0][warp] = a0;
        red[1][warp] = a1;
        red[2][warp] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        R s0 = 0, s1 = 0, s2 = 0;
        for (int w = 0; w < nw; w++) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        const bool ok = s2 > (R)0;
        bc[0] = ok ? s0 / s2 : (R)0;
        bc[1] = ok ? s1 / s2 : (R)0;
        bc[2] = ok ? (R)1 : (R)0;
    }
    __syncthreads();
    alpha = cpx<R>{bc[0], bc[1]};
    return bc[2] > (R)0;
}

// One CTA per block of the given colour.
//   RES = false: the block residual is r_B = v_B (x = 0 everywhere before this sweep);
//   RES = true:  r_B = v_B - (D_W x)_B is formed here from global x (own sites and the
//                neighbours across the block faces, which have the other colour and are
//                not written during this launch).
// colour_grid = true: the grid holds only the blocks of this colour (blocks per direction
// all even); otherwise it holds all blocks and the other colour's CTAs return at once.
template <typename R, typename LT, typename ST, bool RES>
__global__ void __launch_bounds__(kBlock, SapMinBlocks<R>::value) k_sap_block(Geom g, SapGeom sg, const LT *__restrict__ U, const ST *__restrict__ v, ST *x, R m4,
                            int colour, int mr_iters, bool colour_grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = sg.nb;
    // block coordinates of this CTA
    int B[4], rem = blockIdx.x;
    if (colour_grid) {
        const int h3 = sg.nblk[3] / 2;
        const int b3h = rem % h3; rem /= h3;
        B[2] = rem % sg.nblk[2]; rem /= sg.nblk[2];
        B[1] = rem % sg.nblk[1];
        B[0] = rem / sg.nblk[1];
        B[3] = 2 * b3h + ((B[0] + B[1] + B[2] + colour) & 1);
    } else {
        B[3] = rem % sg.nblk[3]; rem /= sg.nblk[3];
        B[2] = rem % sg.nblk[2]; rem /= sg.nblk[2];
        B[1] = rem % sg.nblk[1];
        B[0] = rem / sg.nblk[1];
        if (((B[0] + B[1] + B[2] + B[3]) & 1) != colour) return;   // uniform over the CTA
    }
    ST *s = reinterpret_cast<ST *>(smem_raw);
    LT *u = reinterpret_cast<LT *>(s + SapWords<ST>::spinor * nb);
    // the CTA is padded to whole warps; threads t >= nb hold no site but join the reductions
    const bool act = threadIdx.x < nb;
    const int t = act ? threadIdx.x : 0;
    int l[4], rr = t;
    l[3] = rr % sg.b[3]; rr /= sg.b[3];
    l[2] = rr % sg.b[2]; rr /= sg.b[2];
    l[1] = rr % sg.b[1];
    l[0] = rr / sg.b[1];
    int xg[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) xg[mu] = B[mu] * sg.b[mu] + l[mu];
    const int p = (xg[0] + xg[1] + xg[2] + xg[3]) & 1;
    const int i = eo_index(g, xg);
    // links U_mu(x) of the block sites (forward links; backward ones are the neighbours')
    if (act)
#pragma unroll
        for (int mu = 0; mu < 4; mu++) sm_copy_link(u, nb, mu, t, U, g.Vh, p, i);
    cpx<R> res[12], e[12], q[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
        e[c] = cpx<R>{0, 0};
        res[c] = cpx<R>{0, 0};
        q[c] = cpx<R>{0, 0};
    }
    if (act) {
        load_spinor<R>(v, g.Vh, p, i, res);
        if (RES) {   // res = v - D_W x at this site
            cpx<R> hop[12], own[12], dx[12];
            wilson_hop<R>(g, U, x, p, i, hop);
            load_spinor<R>(x, g.Vh, p, i, own);
            wilson_combine<R>(m4, own, hop, dx);
#pragma unroll
            for (int c = 0; c < 12; c++) res[c] = res[c] - dx[c];
        }
    }
    for (int it = 0; it < mr_iters; it++) {
        if (act) sm_store_sp(s, nb, t, res);
        __syncthreads();
        if (act) block_apply<R, LT, ST>(s, u, nb, t, l, sg.b, sg.stride, m4, q);
        R a0 = 0, a1 = 0, a2 = 0;   // per-site and block sums in the arithmetic type
#pragma unroll
        for (int c = 0; c < 12; c++) {
            a0 += q[c].re * res[c].re + q[c].im * res[c].im;   // Re <q, s>
            a1 += q[c].re * res[c].im - q[c].im * res[c].re;   // Im <q, s>
            a2 += norm2(q[c]);
        }
        cpx<R> alpha;
        if (!mr_alpha<R>(a0, a1, a2, alpha)) break;   // uniform over the CTA
#pragma unroll
        for (int c = 0; c < 12; c++) {
            e[c] = e[c] + alpha * res[c];
            res[c] = res[c] - alpha * q[c];
        }
    }
    __syncthreads();   // every thread of the CTA has finished reading x before any writes it
    if (!act) return;
    cpx<R> xv[12];
    load_spinor<R>(x, g.Vh, p, i, xv);
#pragma unroll
    for (int c = 0; c < 12; c++) xv[c] = xv[c] + e[c];
    store_spinor<R>(x, g.Vh, p, i, xv);
}

// ---------------------------------------------------------------------------------
// Several threads per block site (TPS = 2 or 4). At 16^4 a colour has only 128 blocks of
// 4^4 sites, so the one-thread-per-site kernel runs 8 warps on an SM and the MR loop is
// latency-bound; here thread (k, site) of the CTA, k = threadIdx.x / nbp warp-uniform,
// computes the hops of the directions mu in [k*4/TPS, (k+1)*4/TPS) and owns the C =
// 12/TPS spin-colour components [k*C, (k+1)*C) of the MR state. The partial hopping sums
// are combined through shared memory, summed over k in a fixed order (deterministic).

// The two block-local hops of direction MU (hops that leave the block are dropped).
template <int MU, typename R, typename W>
__device__ __forceinline__ void block_hop_dir(const W *s, const W *u, int nb, int t, const int l[4], const int bx[4],
                                              const int stride[4], cpx<R> acc[12]) {
    if (l[MU] + 1 < bx[MU]) {
        cpx<R> v[12], h0[3], h1[3], a0[3], a1[3], m[3][3];
        sm_load_sp(s, nb, t + stride[MU], v);
        sm_load_link(u, nb, MU, t, m);
        proj_fwd(MU, v, h0, h1);
        su3_mul(m, h0, a0);
        su3_mul(m, h1, a1);
        acc_fwd<false>(MU, acc, a0, a1);
    }
    if (l[MU] > 0) {
        cpx<R> v[12], h0[3], h1[3], a0[3], a1[3], m[3][3];
        sm_load_sp(s, nb, t - stride[MU], v);
        sm_load_link(u, nb, MU, t - stride[MU], m);
        proj_bwd(MU, v, h0, h1);
        su3_dag_mul(m, h0, a0);
        su3_dag_mul(m, h1, a1);
        acc_bwd(MU, acc, a0, a1);
    }
}

template <int TPS, typename R, typename W>
__device__ __forceinline__ void block_hop_part(int k, const W *s, const W *u, int nb, int t, const int l[4],
                                               const int bx[4], const int stride[4], cpx<R> acc[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = cpx<R>{0, 0};
    if (TPS == 2) {
        if (k == 0) {
            block_hop_dir<0, R>(s, u, nb, t, l, bx, stride, acc);
            block_hop_dir<1, R>(s, u, nb, t, l, bx, stride, acc);
        } else {
            block_hop_dir<2, R>(s, u, nb, t, l, bx, stride, acc);
            block_hop_dir<3, R>(s, u, nb, t, l, bx, stride, acc);
        }
    } else {
        switch (k) {
            case 0: block_hop_dir<0, R>(s, u, nb, t, l, bx, stride, acc); break;
            case 1: block_hop_dir<1, R>(s, u, nb, t, l, bx, stride, acc); break;
            case 2: block_hop_dir<2, R>(s, u, nb, t, l, bx, stride, acc); break;
            default: block_hop_dir<3, R>(s, u, nb, t, l, bx, stride, acc); break;
        }
    }
}

// The hops of this thread's directions on the whole lattice (global memory).
template <int TPS, typename R, typename LT, typename ST>
__device__ __forceinline__ void glob_hop_part(int k, const Geom &g, const LT *__restrict__ U, ST in, int p, int i,
                                              const int x[4], cpx<R> acc[12]) {
    if (TPS == 2) {
        if (k == 0) {
            hop_dir<0, true, R>(g, U, in, p, i, x, acc);
            hop_dir<1, false, R>(g, U, in, p, i, x, acc);
        } else {
            hop_dir<2, true, R>(g, U, in, p, i, x, acc);
            hop_dir<3, false, R>(g, U, in, p, i, x, acc);
        }
    } else {
        switch (k) {
            case 0: hop_dir<0, true, R>(g, U, in, p, i, x, acc); break;
            case 1: hop_dir<1, true, R>(g, U, in, p, i, x, acc); break;
            case 2: hop_dir<2, true, R>(g, U, in, p, i, x, acc); break;
            default: hop_dir<3, true, R>(g, U, in, p, i, x, acc); break;
        }
    }
}

// Components [c0, c0 + C) of site (p, i) of an FP32 spinor (complex c is float2 number
// 2 * ((p * 6 + c / 2) * Vh + i) + c % 2 of the float4 array).
template <int C>
__device__ __forceinline__ void load_comps(const float4 *f, int Vh, int p, int i, int c0, cpx<float> o[C]) {
    const float2 *f2 = reinterpret_cast<const float2 *>(f);
#pragma unroll
    for (int e = 0; e < C; e++) {
        const int c = c0 + e;
        const float2 w = f2[2 * ((size_t)(p * 6 + c / 2) * Vh + i) + (c & 1)];
        o[e] = cpx<float>{w.x, w.y};
    }
}
template <int C>
__device__ __forceinline__ void store_comps(float4 *f, int Vh, int p, int i, int c0, const cpx<float> o[C]) {
    float2 *f2 = reinterpret_cast<float2 *>(f);
#pragma unroll
    for (int e = 0; e < C; e++) {
        const int c = c0 + e;
        f2[2 * ((size_t)(p * 6 + c / 2) * Vh + i) + (c & 1)] = make_float2(o[e].re, o[e].im);
    }
}

// Sum over the TPS partial hopping sums of this thread's components: every thread wrote
// its acc[12] to X[k][24][nb]; component c0 + e of the site is summed over k in order.
template <int TPS, int C, typename R>
__device__ __forceinline__ void gather_part(const R *X, int nb, int t, int c0, cpx<R> h[C]) {
#pragma unroll
    for (int e = 0; e < C; e++) {
        const int c = c0 + e;
        R re = X[(2 * c) * nb + t], im = X[(2 * c + 1) * nb + t];
#pragma unroll
        for (int kk = 1; kk < TPS; kk++) {
            re += X[((size_t)kk * 24 + 2 * c) * nb + t];
            im += X[((size_t)kk * 24 + 2 * c + 1) * nb + t];
        }
        h[e] = cpx<R>{re, im};
    }
}
template <typename R>
__device__ __forceinline__ void scatter_part(R *X, int nb, int t, int k, const cpx<R> acc[12]) {
    R *b = X + (size_t)k * 24 * nb + t;
#pragma unroll
    for (int c = 0; c < 12; c++) {
        b[(2 * c) * nb] = acc[c].re;
        b[(2 * c + 1) * nb] = acc[c].im;
    }
}

// FP32 only (the FP64 state would not fit in shared memory for 4^4 blocks). The CTA has
// TPS * nbp threads, nbp = nb rounded up to whole warps (at most 256 sites per block).
template <int TPS, bool RES>
__global__ void __launch_bounds__(256 * TPS, 1)
    k_sap_block_mt(Geom g, SapGeom sg, const float4 *__restrict__ U, const float4 *__restrict__ v, float4 *x, float m4,
                   int colour, int mr_iters, bool colour_grid) {
    using R = float;
    constexpr int C = 12 / TPS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = sg.nb;
    const int nbp = (nb + 31) & ~31;
    int B[4], rem = blockIdx.x;
    if (colour_grid) {
        const int h3 = sg.nblk[3] / 2;
        const int b3h = rem % h3; rem /= h3;
        B[2] = rem % sg.nblk[2]; rem /= sg.nblk[2];
        B[1] = rem % sg.nblk[1];
        B[0] = rem / sg.nblk[1];
        B[3] = 2 * b3h + ((B[0] + B[1] + B[2] + colour) & 1);
    } else {
        B[3] = rem % sg.nblk[3]; rem /= sg.nblk[3];
        B[2] = rem % sg.nblk[2]; rem /= sg.nblk[2];
        B[1] = rem % sg.nblk[1];
        B[0] = rem / sg.nblk[1];
        if (((B[0] + B[1] + B[2] + B[3]) & 1) != colour) return;   // uniform over the CTA
    }
    float4 *s = reinterpret_cast<float4 *>(smem_raw);   // [6][nb] spinor of the block
    float4 *u = s + 6 * nb;                              // [4][3][nb] forward links
    R *X = reinterpret_cast<R *>(u + 12 * nb);           // [TPS][24][nb] partial hopping sums
    const int k = threadIdx.x / nbp;           // warp-uniform
    const int ts = threadIdx.x - k * nbp;
    const bool act = ts < nb;
    const int t = act ? ts : 0;
    const int c0 = k * C;
    int l[4], rr = t;
    l[3] = rr % sg.b[3]; rr /= sg.b[3];
    l[2] = rr % sg.b[2]; rr /= sg.b[2];
    l[1] = rr % sg.b[1];
    l[0] = rr / sg.b[1];
    int xg[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) xg[mu] = B[mu] * sg.b[mu] + l[mu];
    const int p = (xg[0] + xg[1] + xg[2] + xg[3]) & 1;
    const int i = eo_index(g, xg);
    if (act)   // forward links of this thread's directions
#pragma unroll
        for (int mu = 0; mu < 4; mu++)
            if (mu * TPS / 4 == k) sm_copy_link(u, nb, mu, t, U, g.Vh, p, i);
    cpx<R> res[C], e[C], q[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        e[c] = cpx<R>{0, 0};
        res[c] = cpx<R>{0, 0};
        q[c] = cpx<R>{0, 0};
    }
    if (act) load_comps<C>(v, g.Vh, p, i, c0, res);
    if (RES) {   // res = v - D_W x at this site, own components
        if (act) {
            cpx<R> acc[12];
            glob_hop_part<TPS, R>(k, g, U, x, p, i, xg, acc);
            scatter_part(X, nb, t, k, acc);
        }
        __syncthreads();
        if (act) {
            cpx<R> hop[C], own[C];
            gather_part<TPS, C>(X, nb, t, c0, hop);
            load_comps<C>(x, g.Vh, p, i, c0, own);
#pragma unroll
            for (int c = 0; c < C; c++) res[c] = res[c] - (m4 * own[c] + hop[c]);
        }
    }
    for (int it = 0; it < mr_iters; it++) {
        if (act) {   // own components c into the float4 words: complex c is half c % 2 of word c / 2
            float2 *s2 = reinterpret_cast<float2 *>(s);
#pragma unroll
            for (int c = 0; c < C; c++) s2[2 * ((c0 + c) / 2 * nb + t) + ((c0 + c) & 1)] = make_float2(res[c].re, res[c].im);
        }
        __syncthreads();
        if (act) {
            cpx<R> acc[12];
            block_hop_part<TPS, R>(k, s, u, nb, t, l, sg.b, sg.stride, acc);
            scatter_part(X, nb, t, k, acc);
        }
        __syncthreads();
        R a0 = 0, a1 = 0, a2 = 0;
        if (act) {
            cpx<R> hop[C];
            gather_part<TPS, C>(X, nb, t, c0, hop);
#pragma unroll
            for (int c = 0; c < C; c++) {
                q[c] = m4 * res[c] + hop[c];
                a0 += q[c].re * res[c].re + q[c].im * res[c].im;   // Re <q, s>
                a1 += q[c].re * res[c].im - q[c].im * res[c].re;   // Im <q, s>
                a2 += norm2(q[c]);
            }
        }
        cpx<R> alpha;
        if (!mr_alpha<R>(a0, a1, a2, alpha)) break;   // uniform over the CTA
#pragma unroll
        for (int c = 0; c < C; c++) {
            e[c] = e[c] + alpha * res[c];
            res[c] = res[c] - alpha * q[c];
        }
    }
    __syncthreads();   // every thread of the CTA has finished reading x before any writes it
    if (!act) return;
    cpx<R> xv[C];
    load_comps<C>(x, g.Vh, p, i, c0, xv);
#pragma unroll
    for (int c = 0; c < C; c++) xv[c] = xv[c] + e[c];
    store_comps<C>(x, g.Vh, p, i, c0, xv);
}

}  // namespace

// Grants the dynamic shared memory of kernel f once per size (per process).
template <typename K>
static cudaError_t grant_smem(K f, size_t smem, size_t &granted) {
    if (smem <= 48 * 1024 || smem <= granted) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    granted = smem;
    return cudaSuccess;
}

// Launch of one colour's block solves: RES forms the block residual from x in the kernel.
template <typename R, typename LT, typename ST, bool RES>
static cudaError_t launch_blocks(const Geom &g, const SapGeom &sg, const LT *U, const ST *v, ST *x, R m4, int colour,
                                 int mr_iters, bool even, int grid, cudaStream_t st) {
    static size_t granted[3] = {0, 0, 0};
    if constexpr (sizeof(R) == 4) {
        if (sg.tps == 2 || sg.tps == 4) {
            const int nbp = (sg.nb + 31) / 32 * 32;
            const size_t smem = (size_t)sg.nb * (18 * sizeof(float4) + 24 * sg.tps * sizeof(float));
            cudaError_t e;
            if (sg.tps == 2) {
                if ((e = grant_smem(k_sap_block_mt<2, RES>, smem, granted[1])) != cudaSuccess) return e;
                k_sap_block_mt<2, RES><<<grid, 2 * nbp, smem, st>>>(g, sg, U, v, x, m4, colour, mr_iters, even);
            } else {
                if ((e = grant_smem(k_sap_block_mt<4, RES>, smem, granted[2])) != cudaSuccess) return e;
                k_sap_block_mt<4, RES><<<grid, 4 * nbp, smem, st>>>(g, sg, U, v, x, m4, colour, mr_iters, even);
            }
            return cudaGetLastError();
        }
    }
    const size_t smem = (size_t)sg.nb * (SapWords<ST>::spinor * sizeof(ST) + 4 * SapWords<LT>::link * sizeof(LT));
    cudaError_t e;
    if ((e = grant_smem(k_sap_block<R, LT, ST, RES>, smem, granted[0])) != cudaSuccess) return e;
    const int threads = (sg.nb + 31) / 32 * 32;
    k_sap_block<R, LT, ST, RES><<<grid, threads, smem, st>>>(g, sg, U, v, x, m4, colour, mr_iters, even);
    return cudaGetLastError();
}

template <typename R, typename LT, typename ST>
static cudaError_t sap_t(const Geom &g, const SapGeom &sg, const LT *U, const ST *v, ST *x, ST *r, R m0,
                         int cycles, int mr_iters, cudaStream_t st,
                         cudaError_t (*wil)(const Geom &, const LT *, const ST *, ST *, R, int, R, const ST *, R,
                                            cudaStream_t)) {
    cudaError_t e = cudaMemsetAsync(x, 0, (size_t)g.V * 24 * sizeof(R), st);
    if (e != cudaSuccess) return e;
    const int nblocks = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    // with an even number of blocks in every direction the colours alternate across every
    // face (also through the periodic boundary): one colour's blocks can form their own
    // residuals in place and the grid can hold only that colour
    const bool even = !(sg.nblk[0] & 1) && !(sg.nblk[1] & 1) && !(sg.nblk[2] & 1) && !(sg.nblk[3] & 1);
    const int grid = even ? nblocks / 2 : nblocks;
    const R m4 = m0 + (R)4;
    bool x_zero = true;
    for (int cyc = 0; cyc < cycles; cyc++) {
        for (int colour = 0; colour < 2; colour++) {
            if (x_zero) {
                e = launch_blocks<R, LT, ST, false>(g, sg, U, v, x, m4, colour, mr_iters, even, grid, st);
            } else if (even) {
                e = launch_blocks<R, LT, ST, true>(g, sg, U, v, x, m4, colour, mr_iters, even, grid, st);
            } else {
                // r = v - D_W x on the whole lattice, then the block solves from r
                if ((e = wil(g, U, x, r, m0, 0, (R)-1, v, (R)1, st)) != cudaSuccess) return e;
                e = launch_blocks<R, LT, ST, false>(g, sg, U, r, x, m4, colour, mr_iters, even, grid, st);
            }
            count_launches(1);
            if (e != cudaSuccess) return e;
            x_zero = false;
        }
    }
    return cudaSuccess;
}

cudaError_t sap_f32(const Geom &g, const SapGeom &sg, const float4 *U, const float4 *v, float4 *x, float4 *r,
                    float m0, int cycles, int mr_iters, cudaStream_t st) {
    return sap_t<float, float4, float4>(g, sg, U, v, x, r, m0, cycles, mr_iters, st, wilson_f32);
}
cudaError_t sap_f64(const Geom &g, const SapGeom &sg, const double2 *U, const double2 *v, double2 *x, double2 *r,
                    double m0, int cycles, int mr_iters, cudaStream_t st) {
    return sap_t<double, double2, double2>(g, sg, U, v, x, r, m0, cycles, mr_iters, st, wilson_f64);
}

}  // namespace ovl

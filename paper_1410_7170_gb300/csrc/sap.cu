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

// Resident CTAs per SM the block kernel is compiled for: FP32 blocks (98 KB of shared
// memory for 4^4 sites) fit two per SM at 128 registers; FP64 blocks (196 KB) fit one.
template <typename R> struct SapMinBlocks { static constexpr int value = 2; };
template <> struct SapMinBlocks<double> { static constexpr int value = 1; };

// Shared-memory layout (R = arithmetic type): spinor s [24][nb], links [4][18][nb].
template <typename R>
struct SapSmem {
    R *s;
    R *u;
};

template <typename R>
__device__ __forceinline__ void sm_load_sp(const R *s, int nb, int t, cpx<R> v[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) v[c] = cpx<R>{s[(2 * c) * nb + t], s[(2 * c + 1) * nb + t]};
}
template <typename R>
__device__ __forceinline__ void sm_store_sp(R *s, int nb, int t, const cpx<R> v[12]) {
#pragma unroll
    for (int c = 0; c < 12; c++) {
        s[(2 * c) * nb + t] = v[c].re;
        s[(2 * c + 1) * nb + t] = v[c].im;
    }
}
template <typename R>
__device__ __forceinline__ void sm_load_link(const R *u, int nb, int mu, int t, cpx<R> m[3][3]) {
    const R *b = u + (size_t)mu * 18 * nb + t;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int c = 0; c < 3; c++) m[a][c] = cpx<R>{b[(a * 6 + 2 * c) * nb], b[(a * 6 + 2 * c + 1) * nb]};
}

// q = D_BB s at local site t (local coords l, extents bx), links of the block in smem.
template <typename R>
__device__ __forceinline__ void block_apply(const R *s, const R *u, int nb, int t, const int l[4], const int bx[4],
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

template <typename R>
__device__ __forceinline__ void block_sum_sh(double v[3], double *sh) {
    // block-wide sum of 3 doubles, result broadcast to every thread via sh[0..2]
    block_sum<3>(v);
    if (threadIdx.x == 0) {
        sh[0] = v[0];
        sh[1] = v[1];
        sh[2] = v[2];
    }
    __syncthreads();
    v[0] = sh[0];
    v[1] = sh[1];
    v[2] = sh[2];
    __syncthreads();
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
    __shared__ double sh[3];
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
    R *s = reinterpret_cast<R *>(smem_raw);
    R *u = s + 24 * nb;
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
#pragma unroll
    for (int mu = 0; mu < 4 && act; mu++) {
        cpx<R> m[3][3];
        load_link<R>(U, g.Vh, p, mu, i, m);
        R *b = u + (size_t)mu * 18 * nb + t;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                b[(a * 6 + 2 * c) * nb] = m[a][c].re;
                b[(a * 6 + 2 * c + 1) * nb] = m[a][c].im;
            }
    }
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
        if (act) block_apply<R>(s, u, nb, t, l, sg.b, sg.stride, m4, q);
        R a0 = 0, a1 = 0, a2 = 0;   // per-site sums in the arithmetic type, block sums in FP64
#pragma unroll
        for (int c = 0; c < 12; c++) {
            a0 += q[c].re * res[c].re + q[c].im * res[c].im;   // Re <q, s>
            a1 += q[c].re * res[c].im - q[c].im * res[c].re;   // Im <q, s>
            a2 += norm2(q[c]);
        }
        double v[3] = {(double)a0, (double)a1, (double)a2};
        block_sum_sh<R>(v, sh);
        if (!(v[2] > 0.0)) break;   // uniform: every thread holds the block sums
        __syncthreads();            // smem s is rewritten at the top of the next step
        const cpx<R> alpha = cpx<R>{(R)(v[0] / v[2]), (R)(v[1] / v[2])};
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

}  // namespace

template <typename R, typename LT, typename ST>
static cudaError_t sap_t(const Geom &g, const SapGeom &sg, const LT *U, const ST *v, ST *x, ST *r, R m0,
                         int cycles, int mr_iters, cudaStream_t st,
                         cudaError_t (*wil)(const Geom &, const LT *, const ST *, ST *, R, int, R, const ST *, R,
                                            cudaStream_t)) {
    const size_t smem = (size_t)sg.nb * (24 + 4 * 18) * sizeof(R);
    static size_t attr_set[2][2] = {{0, 0}, {0, 0}};   // dynamic shared memory granted, per precision/variant
    const int which = sizeof(R) == 8;
    if (smem > 48 * 1024) {
        cudaError_t e;
        if (smem > attr_set[which][0]) {
            if ((e = cudaFuncSetAttribute(k_sap_block<R, LT, ST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess) {
                cudaGetLastError();
                return e;
            }
            attr_set[which][0] = smem;
        }
        if (smem > attr_set[which][1]) {
            if ((e = cudaFuncSetAttribute(k_sap_block<R, LT, ST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess) {
                cudaGetLastError();
                return e;
            }
            attr_set[which][1] = smem;
        }
    }
    cudaError_t e = cudaMemsetAsync(x, 0, (size_t)g.V * 24 * sizeof(R), st);
    if (e != cudaSuccess) return e;
    const int nblocks = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    // with an even number of blocks in every direction the colours alternate across every
    // face (also through the periodic boundary): one colour's blocks can form their own
    // residuals in place and the grid can hold only that colour
    const bool even = !(sg.nblk[0] & 1) && !(sg.nblk[1] & 1) && !(sg.nblk[2] & 1) && !(sg.nblk[3] & 1);
    const int grid = even ? nblocks / 2 : nblocks;
    const int threads = (sg.nb + 31) / 32 * 32;
    bool x_zero = true;
    for (int cyc = 0; cyc < cycles; cyc++) {
        for (int colour = 0; colour < 2; colour++) {
            if (x_zero) {
                k_sap_block<R, LT, ST, false><<<grid, threads, smem, st>>>(g, sg, U, v, x, m0 + (R)4, colour,
                                                                           mr_iters, even);
            } else if (even) {
                k_sap_block<R, LT, ST, true><<<grid, threads, smem, st>>>(g, sg, U, v, x, m0 + (R)4, colour,
                                                                          mr_iters, even);
            } else {
                // r = v - D_W x on the whole lattice, then the block solves from r
                if ((e = wil(g, U, x, r, m0, 0, (R)-1, v, (R)1, st)) != cudaSuccess) return e;
                k_sap_block<R, LT, ST, false><<<grid, threads, smem, st>>>(g, sg, U, r, x, m0 + (R)4, colour,
                                                                           mr_iters, even);
            }
            count_launches(1);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
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

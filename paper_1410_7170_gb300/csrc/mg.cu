// Two-level aggregation multigrid for D_W: the kernels (see mg.h for the layouts).
//
// Restriction and prolongation run one CTA per block (the aggregate pair of a coarse
// site), one thread per block site. The setup builds the coarse operator column by
// column: for the test vector k restricted to chirality chi (all blocks at once) it
// applies the nine parts of D_W (block-internal, and the hops that cross each of the
// eight block faces) and restricts each result, which gives column (chi, k) of the
// self coupling and of the coupling to each neighbour block. The coarse GMRES keeps its
// Hessenberg matrix and Givens rotations in device memory and runs as a fixed sequence
// of kernels that turn into no-ops once the residual estimate has met the tolerance, so
// a coarse solve needs no host round trip.
#include <math.h>

#include "mg.h"
#include "wilson_site.cuh"

namespace ovl {
namespace {

// Site (p, i) of local site l of block B.
__device__ __forceinline__ void block_site(const Geom &g, const SapGeom &sg, int B, int l, int &p, int &i,
                                           int x[4]) {
    int r = B;
    int bc[4];
    bc[3] = r % sg.nblk[3]; r /= sg.nblk[3];
    bc[2] = r % sg.nblk[2]; r /= sg.nblk[2];
    bc[1] = r % sg.nblk[1];
    bc[0] = r / sg.nblk[1];
    int q = l;
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int lm = q / sg.stride[m];
        q -= lm * sg.stride[m];
        x[m] = bc[m] * sg.b[m] + lm;
    }
    const int s = ((x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
    p = (x[0] + x[1] + x[2] + x[3]) & 1;
    i = s >> 1;
}

// FP32 spinor load through the coherent path, for data the same kernel writes (the
// orthonormalisation rewrites the test vectors in place; load_spinor reads through the
// read-only cache, which is only valid for data no thread writes during the kernel).
__device__ __forceinline__ void load_spinor_rw(const float4 *f, int Vh, int p, int i, cpx<float> s[12]) {
    const float4 *b = f + (size_t)p * 6 * Vh + i;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const float4 v = b[(size_t)c * Vh];
        s[2 * c] = cpx<float>{v.x, v.y};
        s[2 * c + 1] = cpx<float>{v.z, v.w};
    }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// out[B * ob + off + chi * nv + k] = <P_k restricted to aggregate (B, chi), r>: one CTA per
// (block B, test vector k), one thread per block site, one block-wide sum of two complex numbers.
__global__ void __launch_bounds__(256) k_mg_restrict(Geom g, SapGeom sg, const float4 *__restrict__ P, int nv,
                                                     const float4 *__restrict__ r, float2 *__restrict__ out, long ob,
                                                     long off) {
    __shared__ float red[8][4];
    const int B = blockIdx.x, k = blockIdx.y, l = threadIdx.x, lane = l & 31, warp = l >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (l < sg.nb) {
        int p, i, x[4];
        block_site(g, sg, B, l, p, i, x);
        cpx<float> rv[12], pv[12];
        load_spinor<float>(r, g.Vh, p, i, rv);
        load_spinor<float>(P + (long)k * g.V * 6, g.Vh, p, i, pv);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const int h = c < 6 ? 0 : 2;
            acc[h] += pv[c].re * rv[c].re + pv[c].im * rv[c].im;
            acc[h + 1] += pv[c].re * rv[c].im - pv[c].im * rv[c].re;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const float s = warp_sum_f(acc[u]);
        if (lane == 0) red[warp][u] = s;
    }
    __syncthreads();
    if (l < 4) {
        float s = 0.f;
        for (int w = 0; w < nw; w++) s += red[w][l];
        float *o = reinterpret_cast<float *>(out + B * ob + off + (l >> 1) * nv + k);
        o[l & 1] = s;
    }
}

// out (+)= sum_k P_k x_c[B][chi(c)][k]
__global__ void __launch_bounds__(256) k_mg_prolong(Geom g, SapGeom sg, const float4 *__restrict__ P, int nv,
                                                    const float2 *__restrict__ xc, float4 *out, int add) {
    __shared__ float2 xs[2 * kMgMaxNv];
    const int B = blockIdx.x, l = threadIdx.x;
    const int nc = 2 * nv;
    for (int t = l; t < nc; t += blockDim.x) xs[t] = xc[(long)B * nc + t];
    __syncthreads();
    if (l >= sg.nb) return;
    int p, i, x[4];
    block_site(g, sg, B, l, p, i, x);
    cpx<float> o[12];
    if (add) load_spinor<float>(out, g.Vh, p, i, o);
    else
#pragma unroll
        for (int c = 0; c < 12; c++) o[c] = cpx<float>{0.f, 0.f};
    const long vs = (long)g.V * 6;
    for (int k = 0; k < nv; k++) {
        cpx<float> pv[12];
        load_spinor<float>(P + k * vs, g.Vh, p, i, pv);
        const float2 a = xs[k], b = xs[nv + k];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            const float2 z = c < 6 ? a : b;
            o[c].re += pv[c].re * z.x - pv[c].im * z.y;
            o[c].im += pv[c].re * z.y + pv[c].im * z.x;
        }
    }
    store_spinor<float>(out, g.Vh, p, i, o);
}

// out = part of D_W(m0) in (see mg.h), one thread per site
__global__ void __launch_bounds__(256) k_mg_dpart(Geom g, SapGeom sg, const float4 *__restrict__ U,
                                                  const float4 *__restrict__ in, float4 *__restrict__ out, float m4,
                                                  int part) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.V) return;
    int p, i, x[4];
    site_of_thread(t, p, i);
    eo_coords(g, p, i, x);
    const int q = 1 - p;
    cpx<float> acc[12];
    if (part == 0) {
        load_spinor<float>(in, g.Vh, p, i, acc);
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = m4 * acc[c];
    } else {
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = cpx<float>{0.f, 0.f};
    }
#pragma unroll 1
    for (int mu = 0; mu < 4; mu++) {
        int xm = 0, bm = 1, Lm = 1;
#pragma unroll
        for (int m = 0; m < 4; m++)
            if (m == mu) {
                xm = x[m];
                bm = sg.b[m];
                Lm = g.L[m];
            }
        const bool cross_f = (xm + 1) % bm == 0, cross_b = xm % bm == 0;
        const bool do_f = part == 0 ? !cross_f : (part == 1 + 2 * mu && cross_f);
        const bool do_b = part == 0 ? !cross_b : (part == 2 + 2 * mu && cross_b);
        if (do_f) {
            int y[4] = {x[0], x[1], x[2], x[3]};
#pragma unroll
            for (int m = 0; m < 4; m++)
                if (m == mu) y[m] = (xm + 1 == Lm) ? 0 : xm + 1;
            const int j = eo_index(g, y);
            cpx<float> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
            load_spinor<float>(in, g.Vh, q, j, s);
            proj_fwd(mu, s, h0, h1);
            flip_half(h0, h1, mu == 0 && g.antiperiodic && x[0] == g.L[0] - 1);
            load_link<float>(U, g.Vh, p, mu, i, u);
            su3_mul(u, h0, a0);
            su3_mul(u, h1, a1);
            acc_fwd<false>(mu, acc, a0, a1);
        }
        if (do_b) {
            int y[4] = {x[0], x[1], x[2], x[3]};
#pragma unroll
            for (int m = 0; m < 4; m++)
                if (m == mu) y[m] = (xm == 0) ? Lm - 1 : xm - 1;
            const int j = eo_index(g, y);
            cpx<float> s[12], h0[3], h1[3], a0[3], a1[3], u[3][3];
            load_spinor<float>(in, g.Vh, q, j, s);
            proj_bwd(mu, s, h0, h1);
            flip_half(h0, h1, mu == 0 && g.antiperiodic && x[0] == 0);
            load_link<float>(U, g.Vh, q, mu, j, u);
            su3_dag_mul(u, h0, a0);
            su3_dag_mul(u, h1, a1);
            acc_bwd(mu, acc, a0, a1);
        }
    }
    store_spinor<float>(out, g.Vh, p, i, acc);
}

// FP32 spinor word k = p*6*Vh + c*Vh + i holds components 2c, 2c+1: chunks 0-2 are spins 0,1
__global__ void k_mg_chiral_mask(long nw, int Vh, const float4 *__restrict__ v, float4 *__restrict__ out, int chi) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (long)gridDim.x * blockDim.x) {
        const int c = (int)((k / Vh) % 6);
        const bool keep = (c < 3) == (chi == 0);
        out[k] = keep ? v[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Block-wide complex sum (FP32 per thread, FP64 across warps); result valid in all threads.
__device__ __forceinline__ cpx<double> block_csum(float re, float im, double (*sm)[2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    re = warp_sum_f(re);
    im = warp_sum_f(im);
    __syncthreads();
    if (lane == 0) {
        sm[warp][0] = re;
        sm[warp][1] = im;
    }
    __syncthreads();
    double a = 0, b = 0;
    for (int w = 0; w < nw; w++) {
        a += sm[w][0];
        b += sm[w][1];
    }
    return cpx<double>{a, b};
}

// Gram-Schmidt (two passes) of the nv vectors on every aggregate, in place.
__global__ void __launch_bounds__(256) k_mg_orth(Geom g, SapGeom sg, float4 *P, int nv) {
    __shared__ double sm[8][2];
    const int B = blockIdx.x, l = threadIdx.x;
    const bool active = l < sg.nb;
    int p = 0, i = 0, x[4];
    if (active) block_site(g, sg, B, l, p, i, x);
    const long vs = (long)g.V * 6;
    for (int chi = 0; chi < 2; chi++) {
        const int c0 = chi * 6;
        for (int k = 0; k < nv; k++) {
            cpx<float> vk[12];
            if (active) load_spinor_rw(P + k * vs, g.Vh, p, i, vk);
            for (int pass = 0; pass < 2; pass++) {
                for (int j = 0; j < k; j++) {
                    cpx<float> vj[12];
                    float re = 0.f, im = 0.f;
                    if (active) {
                        load_spinor_rw(P + j * vs, g.Vh, p, i, vj);
#pragma unroll
                        for (int c = 0; c < 6; c++) {
                            re += vj[c0 + c].re * vk[c0 + c].re + vj[c0 + c].im * vk[c0 + c].im;
                            im += vj[c0 + c].re * vk[c0 + c].im - vj[c0 + c].im * vk[c0 + c].re;
                        }
                    }
                    const cpx<double> d = block_csum(re, im, sm);
                    if (active) {
                        const float dr = (float)d.re, di = (float)d.im;
#pragma unroll
                        for (int c = 0; c < 6; c++) {
                            const cpx<float> a = vj[c0 + c];
                            vk[c0 + c].re -= dr * a.re - di * a.im;
                            vk[c0 + c].im -= dr * a.im + di * a.re;
                        }
                    }
                }
            }
            float nn = 0.f;
            if (active)
#pragma unroll
                for (int c = 0; c < 6; c++) nn += vk[c0 + c].re * vk[c0 + c].re + vk[c0 + c].im * vk[c0 + c].im;
            const cpx<double> n2 = block_csum(nn, 0.f, sm);
            const float inv = n2.re > 0 ? (float)(1.0 / sqrt(n2.re)) : 0.f;
            if (active) {
                // write back only this chirality's components (the other belongs to the other aggregate)
                cpx<float> full[12];
                load_spinor_rw(P + k * vs, g.Vh, p, i, full);
#pragma unroll
                for (int c = 0; c < 6; c++) full[c0 + c] = inv * vk[c0 + c];
                store_spinor<float>(P + k * vs, g.Vh, p, i, full);
            }
            __syncthreads();
        }
    }
}

// A[b][d] = Dc[b][d] Minv[nbr[b][d]] (column-major nc x nc blocks)
__global__ void __launch_bounds__(256) k_mg_rightprec(const float2 *__restrict__ Dc, const float2 *__restrict__ Minv,
                                                     const int *__restrict__ nbr, float2 *__restrict__ A, int nc) {
    const int bd = blockIdx.x;           // b * 9 + d
    const int n = nbr[bd];
    const float2 *D = Dc + (long)bd * nc * nc;
    const float2 *M = Minv + (long)n * nc * nc;
    float2 *O = A + (long)bd * nc * nc;
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
        const int col = e / nc, row = e % nc;
        float re = 0.f, im = 0.f;
        for (int t = 0; t < nc; t++) {
            const float2 a = D[t * nc + row], b = M[col * nc + t];
            re += a.x * b.x - a.y * b.y;
            im += a.x * b.y + a.y * b.x;
        }
        O[col * nc + row] = make_float2(re, im);
    }
}

constexpr int kCoarseThreads = 9 * 2 * kMgMaxNv;   // one thread per (direction, row)

// y[b] = sum_d Op[b][d] (scale * x[nbr[b][d]]); one CTA per coarse site. Thread (d, row) forms
// the product of one nc x nc block with one neighbour's vector (nc terms); the nine partial
// rows are then summed. Returns the row for threads < nc (others: 0). Every thread calls it.
__device__ __forceinline__ float2 coarse_row(const float2 *__restrict__ Op, const int *__restrict__ nbr,
                                             const float2 *__restrict__ x, float scale, int b, int nc,
                                             float2 (*xs)[2 * kMgMaxNv], float2 (*ps)[2 * kMgMaxNv]) {
    const int t = threadIdx.x;
    const int d = t / nc, row = t - d * nc;
    if (d < 9) {
        const float2 v = x[(long)nbr[b * 9 + d] * nc + row];
        xs[d][row] = make_float2(scale * v.x, scale * v.y);
    }
    __syncthreads();
    if (d < 9) {
        const float2 *O = Op + ((long)b * 9 + d) * nc * nc;
        float re = 0.f, im = 0.f;
        for (int col = 0; col < nc; col++) {
            const float2 a = O[col * nc + row], v = xs[d][col];
            re += a.x * v.x - a.y * v.y;
            im += a.x * v.y + a.y * v.x;
        }
        ps[d][row] = make_float2(re, im);
    }
    __syncthreads();
    float re = 0.f, im = 0.f;
    if (t < nc)
        for (int e = 0; e < 9; e++) {
            re += ps[e][t].x;
            im += ps[e][t].y;
        }
    return make_float2(re, im);
}

__global__ void __launch_bounds__(kCoarseThreads) k_mg_coarse_apply(const float2 *Op, const int *nbr, const float2 *x,
                                                                    float2 *y, int nc) {
    __shared__ float2 xs[9][2 * kMgMaxNv], ps[9][2 * kMgMaxNv];
    const float2 r = coarse_row(Op, nbr, x, 1.f, blockIdx.x, nc, xs, ps);
    if (threadIdx.x < nc) y[(long)blockIdx.x * nc + threadIdx.x] = r;
}

#define HIX(i, j) ((((j) * (kMgMaxSteps + 1)) + (i)) * 2)

// Last-CTA detection (as grid_last_block, local copy for the small coarse grids).
__device__ __forceinline__ bool last_cta(unsigned *counter) {
    __shared__ int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// ||r_c|| -> beta0, g = beta0 e_1, j = 0
__global__ void __launch_bounds__(64) k_mgc_init(MgData mg, int m, double tol) {
    __shared__ double sm[8][2];
    const int b = blockIdx.x, t = threadIdx.x;
    float nn = 0.f;
    if (t < mg.nc) {
        const float2 v = mg.rc[(long)b * mg.nc + t];
        nn = v.x * v.x + v.y * v.y;
    }
    const cpx<double> s = block_csum(nn, 0.f, sm);
    if (t == 0) mg.part[b] = s.re;
    if (last_cta(mg.counter) && t == 0) {
        double tot = 0.0;
        for (int k = 0; k < mg.nb; k++) tot += __ldcg(mg.part + k);
        MgCoarseState *cs = mg.cs;
        const double beta = sqrt(tot);
        cs->m = m;
        cs->j = 0;
        cs->steps = 0;
        cs->tol = tol;
        cs->beta0 = beta;
        cs->done = !(beta > 0.0) ? 1 : 0;
        cs->scale = beta > 0.0 ? (float)(1.0 / beta) : 0.f;
        cs->g[0] = beta;
        cs->g[1] = 0.0;
    }
}

// step j: v_j = scale * src (own block written to V[j]); w = A v_j; H[i][j] = <v_i, w>, i <= j.
// The partial dots of a block need no reduction across threads: w and v_j go to shared memory
// and thread i sums <v_i, w> over the block's nc entries.
__global__ void __launch_bounds__(kCoarseThreads) k_mgc_arnoldi(MgData mg) {
    __shared__ float2 xs[9][2 * kMgMaxNv], ps[9][2 * kMgMaxNv];
    __shared__ float2 ws[2 * kMgMaxNv], vs[2 * kMgMaxNv];
    MgCoarseState *cs = mg.cs;
    if (cs->done) return;
    const int j = cs->j, b = blockIdx.x, t = threadIdx.x, nc = mg.nc;
    const float scale = cs->scale;
    const float2 *src = j == 0 ? mg.rc : mg.w[(j - 1) & 1];
    float2 *w = mg.w[j & 1];
    const long at = (long)b * nc + t;
    if (t < nc) {
        const float2 s = src[at];
        const float2 vj = make_float2(scale * s.x, scale * s.y);
        mg.V[(long)j * mg.ncv + at] = vj;
        vs[t] = vj;
    }
    const float2 r = coarse_row(mg.A, mg.nbr, src, scale, b, nc, xs, ps);
    if (t < nc) {
        w[at] = r;
        ws[t] = r;
    }
    __syncthreads();
    if (t <= j) {
        const float2 *vi = mg.V + (long)t * mg.ncv + (long)b * nc;
        float re = 0.f, im = 0.f;
        for (int e = 0; e < nc; e++) {
            const float2 v = t == j ? vs[e] : vi[e], x = ws[e];
            re += v.x * x.x + v.y * x.y;
            im += v.x * x.y - v.y * x.x;
        }
        mg.part[(2 * t) * mg.nb + b] = re;
        mg.part[(2 * t + 1) * mg.nb + b] = im;
    }
    if (last_cta(mg.counter)) {
        for (int i = t; i <= j; i += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < mg.nb; k++) {
                re += __ldcg(mg.part + (2 * i) * mg.nb + k);
                im += __ldcg(mg.part + (2 * i + 1) * mg.nb + k);
            }
            cs->H[HIX(i, j)] = re;
            cs->H[HIX(i, j) + 1] = im;
        }
    }
}

// step j: w -= sum_i H[i][j] v_i; H[j+1][j] = ||w||; Givens rotation; convergence test
__global__ void __launch_bounds__(64) k_mgc_orth(MgData mg) {
    __shared__ double sm[8][2];
    MgCoarseState *cs = mg.cs;
    if (cs->done) return;
    const int j = cs->j, b = blockIdx.x, t = threadIdx.x, nc = mg.nc;
    float2 *w = mg.w[j & 1];
    const long at = (long)b * nc + t;
    float nn = 0.f;
    if (t < nc) {
        float2 v = w[at];
        for (int i = 0; i <= j; i++) {
            const float hr = (float)cs->H[HIX(i, j)], hi = (float)cs->H[HIX(i, j) + 1];
            const float2 q = mg.V[(long)i * mg.ncv + at];
            v.x -= hr * q.x - hi * q.y;
            v.y -= hr * q.y + hi * q.x;
        }
        w[at] = v;
        nn = v.x * v.x + v.y * v.y;
    }
    const cpx<double> s = block_csum(nn, 0.f, sm);
    if (t == 0) mg.part[b] = s.re;
    if (last_cta(mg.counter) && t == 0) {
        double tot = 0.0;
        for (int k = 0; k < mg.nb; k++) tot += __ldcg(mg.part + k);
        const double h = sqrt(tot);
        double *H = cs->H;
        // earlier rotations on column j
        for (int k = 0; k < j; k++) {
            const double c = cs->cs[k], sr = cs->sn[2 * k], si = cs->sn[2 * k + 1];
            const double ar = H[HIX(k, j)], ai = H[HIX(k, j) + 1], br = H[HIX(k + 1, j)], bi = H[HIX(k + 1, j) + 1];
            // (a, b) <- (c a + s b, -conj(s) a + c b)
            H[HIX(k, j)] = c * ar + (sr * br - si * bi);
            H[HIX(k, j) + 1] = c * ai + (sr * bi + si * br);
            H[HIX(k + 1, j)] = -(sr * ar + si * ai) + c * br;
            H[HIX(k + 1, j) + 1] = -(sr * ai - si * ar) + c * bi;
        }
        // new rotation zeroing H[j+1][j] = h (real)
        const double ar = H[HIX(j, j)], ai = H[HIX(j, j) + 1];
        const double aa = sqrt(ar * ar + ai * ai), nu = sqrt(aa * aa + h * h);
        double c, sr, si;
        if (aa == 0.0) {
            c = 0.0;
            sr = 1.0;
            si = 0.0;
        } else {
            c = aa / nu;
            sr = (ar / aa) * h / nu;   // s = (a / |a|) conj(h) / nu, h real
            si = (ai / aa) * h / nu;
        }
        cs->cs[j] = c;
        cs->sn[2 * j] = sr;
        cs->sn[2 * j + 1] = si;
        H[HIX(j, j)] = c * ar + sr * h;
        H[HIX(j, j) + 1] = c * ai + si * h;
        H[HIX(j + 1, j)] = 0.0;
        H[HIX(j + 1, j) + 1] = 0.0;
        // g_{j+1} = -conj(s) g_j, g_j = c g_j
        const double gr = cs->g[2 * j], gi = cs->g[2 * j + 1];
        cs->g[2 * (j + 1)] = -(sr * gr + si * gi);
        cs->g[2 * (j + 1) + 1] = -(sr * gi - si * gr);
        cs->g[2 * j] = c * gr;
        cs->g[2 * j + 1] = c * gi;
        const double res = sqrt(cs->g[2 * (j + 1)] * cs->g[2 * (j + 1)] + cs->g[2 * (j + 1) + 1] * cs->g[2 * (j + 1) + 1]);
        cs->steps = j + 1;
        if (res <= cs->tol * cs->beta0 || j + 1 >= cs->m || !(h > 0.0)) {
            cs->done = 1;
        } else {
            cs->j = j + 1;
            cs->scale = (float)(1.0 / h);
        }
        if (cs->done) {   // back substitution R y = g over the steps taken
            const int k = cs->steps;
            for (int r = k - 1; r >= 0; r--) {
                double yr = cs->g[2 * r], yi = cs->g[2 * r + 1];
                for (int q = r + 1; q < k; q++) {
                    const double hr = H[HIX(r, q)], hi = H[HIX(r, q) + 1];
                    yr -= hr * cs->y[2 * q] - hi * cs->y[2 * q + 1];
                    yi -= hr * cs->y[2 * q + 1] + hi * cs->y[2 * q];
                }
                const double dr = H[HIX(r, r)], di = H[HIX(r, r) + 1], dd = dr * dr + di * di;
                cs->y[2 * r] = dd > 0 ? (yr * dr + yi * di) / dd : 0.0;
                cs->y[2 * r + 1] = dd > 0 ? (yi * dr - yr * di) / dd : 0.0;
            }
        }
    }
}

// x_c[b] = Minv[b] sum_i y_i V[i][b]
__global__ void __launch_bounds__(64) k_mgc_final(MgData mg) {
    __shared__ float2 u[2 * kMgMaxNv];
    const MgCoarseState *cs = mg.cs;
    const int b = blockIdx.x, t = threadIdx.x, nc = mg.nc;
    const long at = (long)b * nc + t;
    const int k = cs->beta0 > 0.0 ? cs->steps : 0;
    if (t < nc) {
        float re = 0.f, im = 0.f;
        for (int i = 0; i < k; i++) {
            const float yr = (float)cs->y[2 * i], yi = (float)cs->y[2 * i + 1];
            const float2 v = mg.V[(long)i * mg.ncv + at];
            re += yr * v.x - yi * v.y;
            im += yr * v.y + yi * v.x;
        }
        u[t] = make_float2(re, im);
    }
    __syncthreads();
    if (t < nc) {
        const float2 *M = mg.Minv + (long)b * nc * nc;
        float re = 0.f, im = 0.f;
        for (int col = 0; col < nc; col++) {
            const float2 a = M[col * nc + t], v = u[col];
            re += a.x * v.x - a.y * v.y;
            im += a.x * v.y + a.y * v.x;
        }
        mg.xc[at] = make_float2(re, im);
    }
}

inline int round32(int n) { return (n + 31) / 32 * 32; }

}  // namespace

cudaError_t mg_restrict(const Geom &g, const SapGeom &sg, const float4 *P, int nv, const float4 *r, float2 *out,
                        long ob, long off, cudaStream_t st) {
    const int nb = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    k_mg_restrict<<<dim3(nb, nv), round32(sg.nb), 0, st>>>(g, sg, P, nv, r, out, ob, off);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_prolong(const Geom &g, const SapGeom &sg, const float4 *P, int nv, const float2 *xc, float4 *out,
                       bool add, cudaStream_t st) {
    const int nb = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    k_mg_prolong<<<nb, round32(sg.nb), 0, st>>>(g, sg, P, nv, xc, out, add ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_dpart(const Geom &g, const SapGeom &sg, const float4 *U, const float4 *in, float4 *out, float m0,
                     int part, cudaStream_t st) {
    k_mg_dpart<<<plain_grid(g.V), kBlock, 0, st>>>(g, sg, U, in, out, m0 + 4.f, part);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_chiral_mask(const Geom &g, const float4 *v, float4 *out, int chi, cudaStream_t st) {
    const long nw = (long)g.V * 6;
    k_mg_chiral_mask<<<(int)std::min<long>((nw + kBlock - 1) / kBlock, 16L * g.nsm), kBlock, 0, st>>>(nw, g.Vh, v,
                                                                                                      out, chi);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_orthonormalise(const Geom &g, const SapGeom &sg, float4 *P, int nv, cudaStream_t st) {
    const int nb = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    k_mg_orth<<<nb, round32(sg.nb), 0, st>>>(g, sg, P, nv);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_right_precondition(const MgData &mg, cudaStream_t st) {
    k_mg_rightprec<<<mg.nb * 9, 256, 0, st>>>(mg.Dc, mg.Minv, mg.nbr, mg.A, mg.nc);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_coarse_apply(const MgData &mg, const float2 *x, float2 *y, cudaStream_t st) {
    k_mg_coarse_apply<<<mg.nb, kCoarseThreads, 0, st>>>(mg.Dc, mg.nbr, x, y, mg.nc);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t mg_coarse_solve(const MgData &mg, int m, double tol, cudaStream_t st) {
    k_mgc_init<<<mg.nb, 64, 0, st>>>(mg, m, tol);
    for (int j = 0; j < m; j++) {
        k_mgc_arnoldi<<<mg.nb, kCoarseThreads, 0, st>>>(mg);
        k_mgc_orth<<<mg.nb, 64, 0, st>>>(mg);
    }
    k_mgc_final<<<mg.nb, 64, 0, st>>>(mg);
    count_launches(2L * m + 2);
    return cudaGetLastError();
}

}  // namespace ovl

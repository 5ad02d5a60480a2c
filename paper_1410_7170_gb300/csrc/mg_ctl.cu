// Two-level multigrid for D_W: setup and application (host control), and the C-ABI entry
// points that expose them. The kernels are in mg.cu.
//
// Setup (the adaptive setup of the paper's Wilson solver, Sec. 5.1, in its first phase):
//   nv test vectors from start vectors (given, or seeded pseudo-random), each smoothed
//   mg_setup_iters times by v <- v - M_SAP D_W v (the Schwarz smoother applied to D_W x = 0,
//   which damps the components the smoother handles well and leaves the near-kernel ones);
//   orthonormalised on every aggregate; coarse operator D_c = P^H D_W P assembled column by
//   column from the nine parts of D_W; the diagonal blocks of D_c inverted on the host in FP64
//   (Gauss-Jordan with partial pivoting) and D_c M^{-1} formed for the coarse GMRES.
// Application (one iteration of the two-level method as a preconditioner):
//   x = P x_c, x_c ~ D_c^{-1} P^H r by mg_coarse_steps right-preconditioned GMRES steps (stop
//   at mg_coarse_tol); then x += M_SAP (r - D_W x), the Schwarz smoother on the residual.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <vector>

#include "solver.h"

namespace ovl {

namespace {

using cd = std::complex<double>;

// In-place inverse of the n x n complex matrix a (column-major), Gauss-Jordan with partial
// pivoting; false if it is singular to working precision.
bool invert_host(std::vector<cd> &a, int n) {
    std::vector<cd> inv(n * n, cd(0));
    for (int i = 0; i < n; i++) inv[i * n + i] = 1.0;
    auto A = [&](int r, int c) -> cd & { return a[c * n + r]; };
    auto I = [&](int r, int c) -> cd & { return inv[c * n + r]; };
    for (int col = 0; col < n; col++) {
        int piv = col;
        double best = std::abs(A(col, col));
        for (int r = col + 1; r < n; r++)
            if (std::abs(A(r, col)) > best) {
                best = std::abs(A(r, col));
                piv = r;
            }
        if (!(best > 0.0)) return false;
        if (piv != col)
            for (int c = 0; c < n; c++) {
                std::swap(A(piv, c), A(col, c));
                std::swap(I(piv, c), I(col, c));
            }
        const cd d = 1.0 / A(col, col);
        for (int c = 0; c < n; c++) {
            A(col, c) *= d;
            I(col, c) *= d;
        }
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            const cd f = A(r, col);
            if (f == cd(0)) continue;
            for (int c = 0; c < n; c++) {
                A(r, c) -= f * A(col, c);
                I(r, c) -= f * I(col, c);
            }
        }
    }
    a.swap(inv);
    return true;
}

ovl_status mg_check(Ctx *c, int nv) {
    if (nv < 1 || nv > kMgMaxNv) {
        c->err = "mg_nv must be in [1, " + std::to_string(kMgMaxNv) + "]";
        return OVL_EINVAL;
    }
    int vol = 1;
    for (int m = 0; m < 4; m++) {
        const int b = c->p.sap_block[m];
        if (b < 2 || (b & 1) || c->g.L[m] % b || c->g.L[m] / b < 2) {
            c->err = "multigrid: sap_block must be even and leave at least two blocks in every direction";
            return OVL_EINVAL;
        }
        vol *= b;
    }
    if (vol > 256) {
        c->err = "multigrid: sap_block volume must be <= 256 sites";
        return OVL_EINVAL;
    }
    return OVL_OK;
}

ovl_status mg_alloc(Ctx *c, int nv) {
    MgData &mg = c->mg;
    if (mg.P && mg.nv == nv) return OVL_OK;
    if (mg.P) {   // a different number of test vectors: drop the old workspace
        if (mg.graph) cudaGraphExecDestroy(mg.graph);
        void *ptrs[] = {mg.P, mg.Dc, mg.A, mg.Minv, mg.nbr, mg.V, mg.w[0], mg.rc, mg.part, mg.cs, mg.t1};
        for (void *q : ptrs) {
            cudaFree(q);
            c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), q));
        }
        mg = MgData();
    }
    const SapGeom sg = make_sap_geom(c->g, c->p.sap_block);
    mg.nv = nv;
    mg.nc = 2 * nv;
    mg.nb = sg.nblk[0] * sg.nblk[1] * sg.nblk[2] * sg.nblk[3];
    mg.ncv = (long)mg.nb * mg.nc;
    const size_t vs = (size_t)c->g.V * 6 * sizeof(float4);
    const size_t op = (size_t)mg.nb * 9 * mg.nc * mg.nc * sizeof(float2);
    void *b;
    ST(c->alloc(&b, vs * nv));
    mg.P = (float4 *)b;
    ST(c->alloc(&b, op));
    mg.Dc = (float2 *)b;
    ST(c->alloc(&b, op));
    mg.A = (float2 *)b;
    ST(c->alloc(&b, (size_t)mg.nb * mg.nc * mg.nc * sizeof(float2)));
    mg.Minv = (float2 *)b;
    ST(c->alloc(&b, (size_t)mg.nb * 9 * sizeof(int)));
    mg.nbr = (int *)b;
    ST(c->alloc(&b, (size_t)(kMgMaxSteps + 1) * mg.ncv * sizeof(float2)));
    mg.V = (float2 *)b;
    ST(c->alloc(&b, (size_t)2 * mg.ncv * sizeof(float2)));
    mg.w[0] = (float2 *)b;
    mg.w[1] = mg.w[0] + mg.ncv;
    ST(c->alloc(&b, (size_t)2 * mg.ncv * sizeof(float2)));
    mg.rc = (float2 *)b;
    mg.xc = mg.rc + mg.ncv;
    ST(c->alloc(&b, (size_t)2 * (kMgMaxSteps + 2) * mg.nb * sizeof(double) + 256));
    mg.part = (double *)b;
    mg.counter = (unsigned *)((char *)b + (size_t)2 * (kMgMaxSteps + 2) * mg.nb * sizeof(double));
    ST(c->alloc(&b, sizeof(MgCoarseState)));
    mg.cs = (MgCoarseState *)b;
    ST(c->alloc(&b, vs * 5));
    mg.t1 = (float4 *)b;
    mg.t2 = mg.t1 + (size_t)c->g.V * 6;
    mg.t3 = mg.t2 + (size_t)c->g.V * 6;
    mg.tin = mg.t3 + (size_t)c->g.V * 6;
    mg.tout = mg.tin + (size_t)c->g.V * 6;
    CK(cudaMemsetAsync(mg.counter, 0, sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(mg.cs, 0, sizeof(MgCoarseState), c->stream));
    return OVL_OK;
}

}  // namespace

ovl_status mg_setup(Ctx *c, double m0, const double *start, int n_start) {
    const auto t0 = std::chrono::steady_clock::now();
    const int nv = start ? n_start : c->p.mg_nv;
    ST(mg_check(c, nv));
    ST(mg_alloc(c, nv));
    MgData &mg = c->mg;
    mg.ready = false;
    if (mg.graph) {   // the captured application holds the old setup's mass
        cudaGraphExecDestroy(mg.graph);
        mg.graph = nullptr;
    }
    const Geom &g = c->g;
    SapGeom sg = make_sap_geom(g, c->p.sap_block);
    sg.tps = c->sap_tps;
    const long vw = (long)g.V * 6;   // float4 words per FP32 spinor
    cudaStream_t st = c->stream;
    // start vectors
    for (int k = 0; k < nv; k++) {
        float4 *v = mg.P + k * vw;
        if (start) {
            ST(c->import_vec(start + (size_t)k * c->n64, c->io_a));
            CK(spinor_d2f(g, c->io_a, v, st));
        } else {
            CK(fill_random_f32((float *)v, vw * 4, 0x51ed270bu + 7919u * (unsigned)k, st));
        }
    }
    // smoothing: v <- v - M_SAP D_W v
    for (int it = 0; it < c->p.mg_setup_iters; it++)
        for (int k = 0; k < nv; k++) {
            float4 *v = mg.P + k * vw;
            CK(wilson_f32(g, c->U32, v, mg.t1, (float)m0, 0, 1.f, nullptr, 0.f, st));
            CK(sap_f32(g, sg, c->U32, mg.t1, mg.t2, mg.t3, (float)m0, c->p.sap_cycles, c->p.sap_mr_iters, st));
            CK(dev_axpby_f(-1.f, (const float *)mg.t2, 1.f, (float *)v, vw * 4, st));
        }
    CK(mg_orthonormalise(g, sg, mg.P, nv, st));
    // coarse operator, column (chi, k) at a time
    const long ob = 9L * mg.nc * mg.nc;
    for (int chi = 0; chi < 2; chi++)
        for (int k = 0; k < nv; k++) {
            const int col = chi * nv + k;
            CK(mg_chiral_mask(g, mg.P + k * vw, mg.t1, chi, st));
            for (int part = 0; part < 9; part++) {
                CK(mg_dpart(g, sg, c->U32, mg.t1, mg.t2, (float)m0, part, st));
                CK(mg_restrict(g, sg, mg.P, nv, mg.t2, mg.Dc, ob, ((long)part * mg.nc + col) * mg.nc, st));
            }
        }
    // neighbour table of the coarse lattice (block coordinates, periodic)
    std::vector<int> nbr((size_t)mg.nb * 9);
    for (int b = 0; b < mg.nb; b++) {
        int bc[4], r = b;
        for (int m = 3; m >= 0; m--) {
            bc[m] = r % sg.nblk[m];
            r /= sg.nblk[m];
        }
        auto idx = [&](const int q[4]) {
            return ((q[0] * sg.nblk[1] + q[1]) * sg.nblk[2] + q[2]) * sg.nblk[3] + q[3];
        };
        nbr[b * 9] = b;
        for (int m = 0; m < 4; m++) {
            int f[4] = {bc[0], bc[1], bc[2], bc[3]}, k2[4] = {bc[0], bc[1], bc[2], bc[3]};
            f[m] = (bc[m] + 1) % sg.nblk[m];
            k2[m] = (bc[m] + sg.nblk[m] - 1) % sg.nblk[m];
            nbr[b * 9 + 1 + 2 * m] = idx(f);
            nbr[b * 9 + 2 + 2 * m] = idx(k2);
        }
    }
    CK(cudaMemcpyAsync(mg.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    // inverses of the self blocks, on the host in FP64
    const int nc = mg.nc;
    std::vector<float2> self((size_t)mg.nb * nc * nc);
    CK(cudaMemcpy2DAsync(self.data(), (size_t)nc * nc * sizeof(float2), mg.Dc, (size_t)ob * sizeof(float2),
                         (size_t)nc * nc * sizeof(float2), mg.nb, cudaMemcpyDeviceToHost, st));
    ST(c->sync());
    std::vector<cd> a((size_t)nc * nc);
    for (int b = 0; b < mg.nb; b++) {
        for (int e = 0; e < nc * nc; e++) a[e] = cd(self[(size_t)b * nc * nc + e].x, self[(size_t)b * nc * nc + e].y);
        if (!invert_host(a, nc)) {
            c->err = "multigrid setup: a diagonal block of the coarse operator is singular";
            return OVL_EBREAKDOWN;
        }
        for (int e = 0; e < nc * nc; e++)
            self[(size_t)b * nc * nc + e] = make_float2((float)a[e].real(), (float)a[e].imag());
    }
    CK(cudaMemcpyAsync(mg.Minv, self.data(), self.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    CK(mg_right_precondition(mg, st));
    ST(c->sync());
    mg.m0 = m0;
    mg.ready = true;
    mg.setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    mg.coarse_steps = 0;
    mg.applications = 0;
    return OVL_OK;
}

// The kernels of one application, from r to x.
static cudaError_t mg_apply_kernels(Ctx *c, const float4 *r, float4 *x, double m0) {
    MgData &mg = c->mg;
    const Geom &g = c->g;
    SapGeom sg = make_sap_geom(g, c->p.sap_block);
    sg.tps = c->sap_tps;
    cudaStream_t st = c->stream;
    cudaError_t e;
    if ((e = mg_restrict(g, sg, mg.P, mg.nv, r, mg.rc, mg.nc, 0, st)) != cudaSuccess) return e;
    if ((e = mg_coarse_solve(mg, c->p.mg_coarse_steps, c->p.mg_coarse_tol, st)) != cudaSuccess) return e;
    if ((e = mg_prolong(g, sg, mg.P, mg.nv, mg.xc, x, false, st)) != cudaSuccess) return e;
    if ((e = wilson_f32(g, c->U32, x, mg.t1, (float)m0, 0, -1.f, r, 1.f, st)) != cudaSuccess) return e;   // r - D_W x
    if ((e = sap_f32(g, sg, c->U32, mg.t1, mg.t2, mg.t3, (float)m0, c->p.sap_cycles, c->p.sap_mr_iters, st)) !=
        cudaSuccess)
        return e;
    return dev_axpby_f(1.f, (const float *)mg.t2, 1.f, (float *)x, (long)g.V * 24, st);
}

// One application. The application's some 40 short kernels are captured once per setup as a
// CUDA graph on fixed input and output buffers (the caller's vectors are copied in and out),
// so that a Wilson FGMRES iteration pays one graph launch instead of 40 kernel launches.
ovl_status mg_apply_f32(Ctx *c, const float4 *r, float4 *x, double m0) {
    if (!c->mg.ready || c->mg.m0 != m0) ST(mg_setup(c, m0, nullptr, 0));
    MgData &mg = c->mg;
    cudaStream_t st = c->stream;
    const size_t bytes = (size_t)c->g.V * 6 * sizeof(float4);
    if (!c->p.use_graphs) {
        CK(mg_apply_kernels(c, r, x, m0));
        mg.applications++;
        return OVL_OK;
    }
    if (!mg.graph) {
        const long before = launches_total();
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const cudaError_t ce = mg_apply_kernels(c, mg.tin, mg.tout, m0);
        const cudaError_t ee = cudaStreamEndCapture(st, &graph);
        mg.graph_launches = launches_total() - before;
        count_launches(-mg.graph_launches);   // captured, not run
        CK(ce);
        CK(ee);
        const cudaError_t ie = cudaGraphInstantiate(&mg.graph, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
    }
    CK(cudaMemcpyAsync(mg.tin, r, bytes, cudaMemcpyDeviceToDevice, st));
    CK(cudaGraphLaunch(mg.graph, st));
    count_launches(mg.graph_launches);
    CK(cudaMemcpyAsync(x, mg.tout, bytes, cudaMemcpyDeviceToDevice, st));
    mg.applications++;
    return OVL_OK;
}

}  // namespace ovl

using namespace ovl;

extern "C" ovl_status ovl_mg_setup(ovl_ctx *ctx, double m0, const double *start, int n_start) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (!isfinite(m0) || (start && n_start < 1)) {
        c->err = "ovl_mg_setup: need finite m0 and n_start >= 1 with start vectors";
        return OVL_EINVAL;
    }
    if (!c->sap_tuned) {
        ST(c->autotune_sap());
        c->sap_tuned = true;
    }
    return mg_setup(c, m0, start, n_start);
}

extern "C" ovl_status wilson_mg_apply(ovl_ctx *ctx, double *out, const double *in, double m0) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (!out || !in || !isfinite(m0)) {
        c->err = "wilson_mg_apply: NULL vector or non-finite m0";
        return OVL_EINVAL;
    }
    ST(mg_check(c, c->mg.ready ? c->mg.nv : c->p.mg_nv));
    if (!c->sap_tuned) {
        ST(c->autotune_sap());
        c->sap_tuned = true;
    }
    ST(c->import_vec(in, c->io_a));
    ST(ensure_f32_buffers(c));
    CK(spinor_d2f(c->g, c->io_a, (float4 *)c->f_a, c->stream));
    ST(mg_apply_f32(c, (const float4 *)c->f_a, (float4 *)c->f_b, m0));
    CK(spinor_f2d(c->g, (const float4 *)c->f_b, c->io_b, c->stream));
    return c->export_vec(c->io_b, out);
}

extern "C" ovl_status ovl_mg_info(const ovl_ctx *ctx, int *nv, int *coarse_sites, int *last_coarse_steps,
                                  double *setup_s) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (nv) *nv = c->mg.ready ? c->mg.nv : 0;
    if (coarse_sites) *coarse_sites = c->mg.ready ? c->mg.nb : 0;
    if (setup_s) *setup_s = c->mg.setup_s;
    if (last_coarse_steps) {
        *last_coarse_steps = 0;
        if (c->mg.ready) {
            int s = 0;
            if (cudaMemcpy(&s, &c->mg.cs->steps, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return OVL_ECUDA;
            }
            *last_coarse_steps = s;
        }
    }
    return OVL_OK;
}

// C-ABI entry points and the host-side control of the solvers.
//
//   ovl_create   gauge upload/compression, spectral bounds of |Q| by Lanczos on Q^2,
//                Zolotarev coefficients, optional low-mode deflation, sigma_min of
//                Eq. (default_m) by Lanczos on Q(0)^2 (Sec. 5.1)
//   wilson_apply D_W(m0) (Eq. Wilson-Dirac)
//   sign_apply   sign(Q) by Zolotarev + multishift CG, or by the restarted Krylov method
//                of Sec. 5.2 (krylov.cu)
//   ovl_apply    D_N = rho I + Gamma5 sign(Q) (Eq. overlap_def)
//   ovl_solve    GMRES(m) / FGMRES(m) on D_N psi = eta (Eq. linsys, Sec. 5.1-5.3)
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <complex>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ovl.h"
#include "internal.h"
#include "sap.h"
#include "solver.h"

using namespace ovl;

static thread_local std::string g_create_error;

void ovl::set_thread_error(const std::string &msg) { g_create_error = msg; }

// ------------------------------------------------------------------ defaults
extern "C" ovl_status ovl_params_default(ovl_params *p) {
    if (!p) return OVL_EINVAL;
    memset(p, 0, sizeof(*p));
    p->tol_outer = 1e-8;       // Table 2
    p->restart = 100;          // Table 2
    p->relax = 1;              // Sec. 5.2
    p->relax_factor = 1e-2;    // Table 2
    p->n_poles = 20;
    p->lambda_min = 0.0;
    p->lambda_max = 0.0;
    p->sign_tol = 1e-12;
    p->precond = OVL_PREC_NONE;
    p->m0_prec = NAN;          // m0^def (Eq. default_m)
    p->eps_prec = 1e-1;        // Table 2
    p->eps_inner = 1e-2;       // Table 3 (with preconditioning)
    p->restart_inner = 100;    // Table 3
    p->max_inner = 200;
    p->precision = OVL_FP64;
    p->antiperiodic = 1;
    p->max_iter = 5000;
    p->max_ms_iter = 20000;
    for (int m = 0; m < 4; m++) p->sap_block[m] = 4;
    p->sap_cycles = 2;
    p->sap_mr_iters = 6;
    p->prec_restart = 32;
    p->prec_max_iter = 64;
    p->rhs_block = 4;
    p->use_graphs = 1;
    p->check_every = 8;
    p->stencil_tps = 0;
    p->sap_tps = 0;
    p->adaptive_poles = 1;
    p->n_deflate = 0;
    p->deflate_tol = 1e-13;
    p->sign_method = OVL_SIGN_ZOLOTAREV;
    p->krylov_m = 40;
    p->krylov_keep = 8;
    p->ff_outer = 1;
    p->max_seconds = 0.0;
    p->wilson_mg = 0;
    p->mg_nv = 12;
    p->mg_setup_iters = 4;
    p->mg_coarse_steps = 16;
    p->mg_coarse_tol = 0.1;
    p->m0_adapt = 0;
    p->mrhs_kernel = 0;
    return OVL_OK;
}

static ovl_status validate_params(const ovl_params &p, const int L[4], std::string &err) {
    char buf[256];
    if (!(p.tol_outer > 0 && p.tol_outer < 1)) { err = "tol_outer must be in (0,1)"; return OVL_EINVAL; }
    if (p.restart < 2 || p.restart > 120) { err = "restart must be in [2,120]"; return OVL_EINVAL; }
    if (p.restart_inner < 2 || p.restart_inner > 120) { err = "restart_inner must be in [2,120]"; return OVL_EINVAL; }
    if (p.prec_restart < 2 || p.prec_restart > 120) { err = "prec_restart must be in [2,120]"; return OVL_EINVAL; }
    if (p.n_poles < 1 || p.n_poles > kMaxPoles) {
        snprintf(buf, sizeof buf, "n_poles must be in [1,%d]", kMaxPoles);
        err = buf;
        return OVL_EINVAL;
    }
    if (p.lambda_min < 0 || p.lambda_max < 0 || (p.lambda_min > 0 && !(p.lambda_max > p.lambda_min))) {
        err = "need 0 < lambda_min < lambda_max (or both 0 to estimate)";
        return OVL_EINVAL;
    }
    if (p.precond < 0 || p.precond > 2) { err = "precond must be 0, 1 or 2"; return OVL_EINVAL; }
    if (p.precision < 0 || p.precision > 3) { err = "precision must be 0, 1, 2 or 3"; return OVL_EINVAL; }
    if (p.max_iter < 1 || p.max_ms_iter < 1 || p.check_every < 1) { err = "iteration caps must be >= 1"; return OVL_EINVAL; }
    if (p.rhs_block < 1 || p.rhs_block > 12) { err = "rhs_block must be in [1,12]"; return OVL_EINVAL; }
    if (p.stencil_tps != 0 && p.stencil_tps != 1 && p.stencil_tps != 4) { err = "stencil_tps must be 0, 1 or 4"; return OVL_EINVAL; }
    if (p.sap_tps != 0 && p.sap_tps != 1 && p.sap_tps != 2 && p.sap_tps != 4) { err = "sap_tps must be 0, 1, 2 or 4"; return OVL_EINVAL; }
    if (p.adaptive_poles != 0 && p.adaptive_poles != 1) { err = "adaptive_poles must be 0 or 1"; return OVL_EINVAL; }
    if (p.n_deflate < 0 || p.n_deflate > 48) { err = "n_deflate must be in [0, 48]"; return OVL_EINVAL; }
    if (p.n_deflate > 0 && !(p.deflate_tol > 0 && p.deflate_tol <= 1e-3)) { err = "deflate_tol must be in (0, 1e-3]"; return OVL_EINVAL; }
    if (p.sign_method != OVL_SIGN_ZOLOTAREV && p.sign_method != OVL_SIGN_KRYLOV) { err = "sign_method must be 0 or 1"; return OVL_EINVAL; }
    if (p.krylov_m < 4 || p.krylov_m > 120) { err = "krylov_m must be in [4,120]"; return OVL_EINVAL; }
    if (p.krylov_keep < 0 || p.krylov_keep > p.krylov_m - 2) { err = "krylov_keep must be in [0, krylov_m - 2]"; return OVL_EINVAL; }
    if (p.ff_outer != 0 && p.ff_outer != 1) { err = "ff_outer must be 0 or 1"; return OVL_EINVAL; }
    if (!(p.max_seconds >= 0)) { err = "max_seconds must be >= 0"; return OVL_EINVAL; }
    if (p.wilson_mg != 0 && p.wilson_mg != 1) { err = "wilson_mg must be 0 or 1"; return OVL_EINVAL; }
    if (p.mg_nv < 1 || p.mg_nv > kMgMaxNv) { err = "mg_nv must be in [1, 24]"; return OVL_EINVAL; }
    if (p.mg_setup_iters < 0 || p.mg_setup_iters > 100) { err = "mg_setup_iters must be in [0, 100]"; return OVL_EINVAL; }
    if (p.mg_coarse_steps < 1 || p.mg_coarse_steps > kMgMaxSteps) { err = "mg_coarse_steps must be in [1, 64]"; return OVL_EINVAL; }
    if (!(p.mg_coarse_tol >= 0 && p.mg_coarse_tol < 1)) { err = "mg_coarse_tol must be in [0, 1)"; return OVL_EINVAL; }
    if (p.m0_adapt != 0 && p.m0_adapt != 1) { err = "m0_adapt must be 0 or 1"; return OVL_EINVAL; }
    if (p.mrhs_kernel < 0 || p.mrhs_kernel > 3) { err = "mrhs_kernel must be in [0, 3]"; return OVL_EINVAL; }
    if (p.wilson_mg) {
        for (int m = 0; m < 4; m++)
            if (p.sap_block[m] < 2 || (p.sap_block[m] & 1) || L[m] % p.sap_block[m] || L[m] / p.sap_block[m] < 2) {
                err = "wilson_mg needs even sap_block extents leaving at least two blocks per direction";
                return OVL_EINVAL;
            }
    }
    for (int m = 0; m < 4 && p.precond != OVL_PREC_NONE; m++) {
        if (p.sap_block[m] < 2 || (p.sap_block[m] & 1) || L[m] % p.sap_block[m]) {
            err = "sap_block must be even and divide the lattice extent";
            return OVL_EINVAL;
        }
    }
    if (p.precond != OVL_PREC_NONE) {
        const int nb = p.sap_block[0] * p.sap_block[1] * p.sap_block[2] * p.sap_block[3];
        if (nb > 256) { err = "sap_block volume must be <= 256 sites"; return OVL_EINVAL; }
        if (p.sap_cycles < 1 || p.sap_mr_iters < 1) { err = "sap_cycles, sap_mr_iters must be >= 1"; return OVL_EINVAL; }
    }
    return OVL_OK;
}

// ------------------------------------------------------------------ helpers
static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ovl_status Ctx::alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = "device allocation of " + std::to_string(bytes) + " bytes failed";
        *p = nullptr;
        return OVL_ENOMEM;
    }
    allocs.push_back(*p);
    bytes_held += bytes;
    return OVL_OK;
}

Ctx::~Ctx() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto &gr : graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    if (mg.graph) cudaGraphExecDestroy(mg.graph);
    for (int w = 0; w < 3; w++)
        if (ev_ready[w])
            for (int k = 0; k < 4; k++) cudaEventDestroy(ev[w][k]);
    for (void *p : allocs) cudaFree(p);
    if (h_pinned) cudaFreeHost(h_pinned);
    if (own_stream && stream) cudaStreamDestroy(stream);
}

ovl_status Ctx::sync() {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        err = std::string("CUDA: ") + cudaGetErrorString(e);
        return OVL_ECUDA;
    }
    return OVL_OK;
}

// Device scalars -> host (pinned), synchronising the stream.
ovl_status Ctx::fetch(const double *d, int n, double *h) {
    Ctx *c = this;
    CK(cudaMemcpyAsync(h_scal, d, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    ST(sync());
    memcpy(h, h_scal, n * sizeof(double));
    return OVL_OK;
}

ovl_status Ctx::norm2_d(const double *x, double *out) {
    Ctx *c = this;
    CK(dev_norm2(x, n64, d_scal, rs, stream));
    return fetch(d_scal, 1, out);
}
ovl_status Ctx::norm2_f(const float *x, double *out) {
    Ctx *c = this;
    CK(dev_norm2_f(x, n64, d_scal, rs, stream));
    return fetch(d_scal, 1, out);
}

// Copy a boundary vector (host or device, lexicographic) into an internal FP64 eo vector.
ovl_status Ctx::import_vec(const double *src, double2 *dst) {
    Ctx *c = this;
    const double *lex = src;
    if (!is_device_ptr(src)) {
        CK(cudaMemcpyAsync(io_lex, src, n64 * sizeof(double), cudaMemcpyHostToDevice, stream));
        lex = io_lex;
    }
    CK(pack_spinor_f64(g, dst, lex, stream));
    CK(cudaMemsetAsync(d_flag, 0, sizeof(int), stream));
    CK(dev_nonfinite((const double *)dst, n64, d_flag, stream));
    int h = 0;
    CK(cudaMemcpyAsync(h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
    ST(sync());
    h = *h_flag;
    if (h) {
        err = "input vector holds NaN or Inf";
        return OVL_EINVAL;
    }
    return OVL_OK;
}

ovl_status Ctx::export_vec(const double2 *src, double *dst) {
    Ctx *c = this;
    if (is_device_ptr(dst)) {
        CK(unpack_spinor_f64(g, dst, src, stream));
        return sync();
    }
    CK(unpack_spinor_f64(g, io_lex, src, stream));
    CK(cudaMemcpyAsync(dst, io_lex, n64 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    return sync();
}

// ------------------------------------------------------------------ multishift sign
// Zolotarev degree for a sign application of relative accuracy tol: the smallest n <=
// n_poles whose uniform approximation error delta(k, n) is at most tol / 10, so that the
// rational approximation stays an order below the multishift CG's own error (with
// adaptive_poles = 0: always n_poles). Fewer poles mean fewer shifted directions to
// update and a larger smallest shift (faster CG convergence).
int Ctx::pick_poles(double tol) const {
    if (!p.adaptive_poles) return npole;
    for (int n = 1; n < npole; n++)
        if (zs_delta[n - 1] <= 0.1 * tol) return n;
    return npole;
}

// Multishift state of degree n for tolerance tol.
void Ctx::fill_poles(MsState &s, int n, double tol) const {
    memset(&s, 0, sizeof(MsState));
    s.n = n;
    s.tol = tol;
    s.alpha_prev = 1.0;
    s.beta_prev = 0.0;
    const std::vector<double> &a = zs_a[n - 1], &c = zs_c[n - 1];
    const double d0 = zs_d0[n - 1];
    // The residual r_l of shift l adds (d0/lmin) a_l lmin^2 Q (Q^2 + sigma_l)^{-1} r_l to sign(Q) b.
    // With |Q| in [lmin, lmax] (the interval the rational approximation assumes) its norm is at
    // most d0 |a_l| g_l ||r_l||, g_l = max of x/(x^2 + c_l) over x in [1, lmax/lmin]. Shift l is
    // dropped once that bound is below its share of tol ||b||: half for the smallest shift (the
    // slowest to converge), the other half split evenly; the shares sum to 1.
    const double K = lam_max / lam_min;
    int l_small = 0;
    for (int l = 1; l < n; l++)
        if (c[l] < c[l_small]) l_small = l;
    for (int l = 0; l < n; l++) {
        s.sigma[l] = lam_min * lam_min * c[l];
        s.w[l] = a[l] * lam_min * lam_min;
        const double rc = sqrt(c[l]);
        const double g = rc <= 1.0 ? 1.0 / (1.0 + c[l]) : (rc >= K ? K / (K * K + c[l]) : 0.5 / rc);
        const double share = n == 1 ? 1.0 : (l == l_small ? 0.5 : 0.5 / (n - 1));
        s.crit[l] = d0 * fabs(a[l]) * g / share;
        s.zeta[l] = 1.0;
        s.zeta_prev[l] = 1.0;
        s.active[l] = 1;
    }
}

// Fills the multishift state for tolerance tol and uploads it; *n_out = the degree used.
ovl_status Ctx::ms_setup(MsState *d_state, double tol, int *n_out) {
    Ctx *c = this;
    const int n = pick_poles(tol);
    fill_poles(*h_ms, n, tol);
    h_ms->hist = prof ? d_hist : nullptr;
    h_ms->hist_cap = prof ? hist_cap : 0;
    CK(cudaMemcpyAsync(d_state, h_ms, sizeof(MsState), cudaMemcpyHostToDevice, stream));
    *n_out = n;
    return OVL_OK;
}

// Polls the device state every check_every iterations; graphs replay the chunk.
// With instrumentation on, event records around the first three kernels of every
// iteration are part of the queued work (event record nodes inside graphs) and the
// device logs how many shifts each iteration updated, so per-kernel durations and
// algorithmic bytes come from the same launches that do the work.
template <typename Iter>
ovl_status Ctx::ms_run(MsState *d_state, int which, int slot, double shift_bytes, bool fused, Iter iter_fn,
                       int *iters_out) {
    Ctx *c = this;
    const int chunk = std::min(p.check_every, kMaxChunk);
    const int sample = chunk / 2;   // the iteration of every chunk whose kernels are timed
    const double rbytes = which == 1 ? 4.0 : 8.0;   // bytes per real: FP32 slot 4, FP64 and float-float 8
    int done_iters = 0, iter_before = 0;
    GraphSlot &gs = graphs[slot];
    if (prof && !ev_ready[which]) {
        for (int k = 0; k < 4; k++) CK(cudaEventCreate(&ev[which][k]));
        ev_ready[which] = true;
    }
    if (gs.exec && (gs.chunk != chunk || gs.prof != prof)) {
        cudaGraphExecDestroy(gs.exec);
        gs.exec = nullptr;
    }
    while (true) {
        if (p.use_graphs) {
            if (!gs.exec) {
                cudaGraph_t graph;
                set_launch_counting(false);
                CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaSuccess;
                for (int k = 0; k < chunk && ce == cudaSuccess; k++)
                    ce = iter_fn(prof && k == sample ? ev[which] : nullptr, cudaEventRecordExternal);
                cudaError_t ee = cudaStreamEndCapture(stream, &graph);
                set_launch_counting(true);
                CK(ce);
                CK(ee);
                cudaError_t ie = cudaGraphInstantiate(&gs.exec, graph, 0);
                cudaGraphDestroy(graph);
                CK(ie);
                gs.chunk = chunk;
                gs.prof = prof;
            }
            CK(cudaGraphLaunch(gs.exec, stream));
            count_launches(3L * chunk);
        } else {
            for (int k = 0; k < chunk; k++) CK(iter_fn(prof && k == sample ? ev[which] : nullptr, 0u));
        }
        done_iters += chunk;
        CK(cudaMemcpyAsync(h_ms_small, d_state, 4 * sizeof(int), cudaMemcpyDeviceToHost, stream));
        if (prof) CK(cudaMemcpyAsync(h_hist, d_hist + iter_before, chunk * sizeof(int), cudaMemcpyDeviceToHost,
                                     stream));
        ST(sync());
        const int iter = h_ms_small[1], done = h_ms_small[2], status = h_ms_small[3];
        if (prof) {
            const int ran = std::min(chunk, iter - iter_before);
            const double V = (double)g.V;
            ProfAcc &pa = pacc[which];
            // algorithmic reals per site: Q p: p, 4 links x 12, t; residual: t, links, p, r in/out;
            // shifts: r, y in/out, each updated p_l in/out. Fused form: the residual kernel also
            // moves y in/out and the p_l (l >= 1), the third kernel r, p_0 in/out.
            const double qb = 96.0 * V * rbytes;
            for (int k = 0; k < ran; k++) {
                const double rb = fused ? (192.0 * rbytes + shift_bytes * (h_hist[k] - 1)) * V : 144.0 * V * rbytes;
                const double sb = fused ? 72.0 * rbytes * V : (72.0 * rbytes + shift_bytes * h_hist[k]) * V;
                pa.n++;
                pa.q_bytes += qb;
                pa.r_bytes += rb;
                pa.s_bytes += sb;
                if (k != sample) continue;
                float a = 0, b = 0, d = 0;
                if (cudaEventElapsedTime(&a, ev[which][0], ev[which][1]) != cudaSuccess ||
                    cudaEventElapsedTime(&b, ev[which][1], ev[which][2]) != cudaSuccess ||
                    cudaEventElapsedTime(&d, ev[which][2], ev[which][3]) != cudaSuccess) {
                    cudaGetLastError();
                    pa.valid = false;
                    continue;
                }
                pa.q_ms += a; pa.r_ms += b; pa.s_ms += d;
                pa.q_t++; pa.r_t++; pa.s_t++;
                pa.q_tb += qb; pa.r_tb += rb; pa.s_tb += sb;
            }
        }
        iter_before = iter;
        if (status) {
            err = "multishift CG breakdown (non-finite or non-positive scalar)";
            return OVL_EBREAKDOWN;
        }
        if (!done && past_deadline()) return OVL_ETIMEOUT;
        if (done) {
            *iters_out = iter;
            return OVL_OK;
        }
        if (iter >= p.max_ms_iter || done_iters > p.max_ms_iter + chunk) {
            *iters_out = iter;
            err = "multishift CG reached max_ms_iter";
            return OVL_ENOCONV;
        }
    }
}

// y = b + sum_l w_l (Q^2+sigma_l)^{-1} b in FP64; then
//   mode 0: out = (d0/lmin) gamma5 D_W y = sign(Q) b
//   mode 1: out = rho b + (d0/lmin) D_W y   = D_N b
ovl_status Ctx::sign64(const double2 *b, double2 *out, double tol, int mode) {
    if (p.sign_method == OVL_SIGN_KRYLOV) return sign64_krylov(b, out, tol, mode);
    PhaseClock pclk(this, &t_sign64);
    Ctx *c = this;
    ST(ensure_ms64());
    // with deflation the multishift sees Pi b only; the deflated eigenpairs are added exactly
    std::vector<double> dc;
    const double2 *bm = b;
    if (ndefl) {
        ST(defl_project64(b, defl_tmp64, dc));
        bm = defl_tmp64;
    }
    int n;
    ST(ms_setup(ms64_state, tol, &n));
    CK(ms_init_f64(g, n, ms64_state, ms64, bm, rs, stream));
    int iters = 0;
    auto fn = [&](cudaEvent_t *e, unsigned f) { return ms_iter_f64(g, U64, m0_ker, ms64_state, ms64, rs, stream, e, f); };
    // at the iteration cap the output is still formed from the last iterate (status ENOCONV)
    const ovl_status ms = ms_run(ms64_state, 0, 0, 48.0 * 8.0, false, fn, &iters);
    if (ms != OVL_OK && ms != OVL_ENOCONV) return ms;
    stat_ms64 += iters;
    const double sc = zs_d0[n - 1] / lam_min;
    if (mode == 0) CK(wilson_f64(g, U64, ms64.y, out, m0_ker, 1, sc, nullptr, 0.0, stream));
    else CK(wilson_f64(g, U64, ms64.y, out, m0_ker, 0, sc, b, rho, stream));
    if (ndefl) ST(defl_add64(dc, out, mode));
    return ms;
}

// y = b + sum_l w_l (Q^2+sigma_l)^{-1} b in float-float arithmetic (ff.cuh) on the FP32
// pipes, for the sign applications that need FP64 accuracy; b, out are FP64 even-odd
// spinors and the result has the same form as sign64's. The multishift vectors and links
// are float-float; the Zolotarev coefficients and the CG scalars stay FP64 on the device.
ovl_status Ctx::sign_ff(const double2 *b, double2 *out, double tol, int mode) {
    if (p.sign_method == OVL_SIGN_KRYLOV) return sign64_krylov(b, out, tol, mode);
    PhaseClock pclk(this, &t_sign64);
    Ctx *c = this;
    ST(ensure_msff());
    std::vector<double> dc;
    const double2 *bm = b;
    if (ndefl) {
        ST(defl_project64(b, defl_tmp64, dc));
        bm = defl_tmp64;
    }
    const long words = (long)g.V * 12;
    int n;
    ST(ms_setup(msff_state, tol, &n));
    // b in float-float into t (t is overwritten by the first iteration's Q p)
    CK(dev_d2ff(bm, msff.t, words, stream));
    CK(ms_init_ff(g, n, msff_state, msff, msff.t, rs, stream));
    int iters = 0;
    auto fn = [&](cudaEvent_t *e, unsigned f) { return ms_iter_ff(g, Uff, m0_ker, msff_state, msff, rs, stream, e, f); };
    const ovl_status ms = ms_run(msff_state, 2, 5, 48.0 * 8.0, false, fn, &iters);
    if (ms != OVL_OK && ms != OVL_ENOCONV) return ms;
    stat_msff += iters;
    const double sc = zs_d0[n - 1] / lam_min;
    // s = (d0/lmin) [gamma5] D_W y in float-float, then FP64; D_N b = rho b + s without gamma5
    CK(wilson_ff(g, Uff, msff.y, msff.t, m0_ker, mode == 0, sc, nullptr, 0.0, stream));
    CK(dev_ff2d(msff.t, out, words, stream));
    if (mode == 1) CK(dev_axpby(rho, (const double *)b, 1.0, (double *)out, 2 * words, stream));
    if (ndefl) ST(defl_add64(dc, out, mode));
    return ms;
}

ovl_status Ctx::ensure_ff_links() {
    Ctx *c = this;
    if (Uff) return OVL_OK;
    const long words = (long)g.V * 4 * kLink64Words;
    ST(alloc((void **)&Uff, (size_t)words * sizeof(ffw)));
    CK(dev_d2ff(U64, Uff, words, stream));
    return OVL_OK;
}

ovl_status Ctx::ensure_16(bool bf16) {
    Ctx *c = this;
    const int k = bf16 ? 1 : 0;
    if (!U16[k]) {
        ST(alloc(&U16[k], (size_t)g.V * 4 * 3 * sizeof(uint2)));
        CK(links_to16(g, U32, U16[k], bf16, stream));
    }
    if (!h16a) {
        void *buf;
        const size_t sp = (size_t)g.V * 3 * sizeof(uint4), nb = (size_t)g.V * sizeof(float);
        ST(alloc(&buf, 2 * sp + 2 * nb));
        h16a = (uint4 *)buf;
        h16b = (uint4 *)((char *)buf + sp);
        h16na = (float *)((char *)buf + 2 * sp);
        h16nb = (float *)((char *)buf + 2 * sp + nb);
    }
    return OVL_OK;
}

ovl_status Ctx::ensure_msff() {
    ST(ensure_ff_links());
    if (msff.p) return OVL_OK;
    void *buf;
    if (!msff_state) {
        ST(alloc(&buf, sizeof(MsState)));
        msff_state = (MsState *)buf;
    }
    const long words = (long)g.V * 12;   // ffw per vector
    ST(alloc(&buf, (size_t)words * sizeof(ffw) * (npole + 3)));
    ffw *f = (ffw *)buf;
    msff.r = f;
    msff.t = f + words;
    msff.y = f + 2 * words;
    msff.p = f + 3 * words;
    msff.stride = words;
    return OVL_OK;
}

ovl_status Ctx::sign_outer(const double2 *b, double2 *out, double tol, int mode) {
    if (p.precision != OVL_FP64 && p.ff_outer) return sign_ff(b, out, tol, mode);
    return sign64(b, out, tol, mode);
}

ovl_status Ctx::sign_outer_batch(const double2 *b, double2 *out, int nrhs, const double *tol, int mode) {
    if (!(p.precision != OVL_FP64 && p.ff_outer)) return sign64_batch(b, out, nrhs, tol, mode);
    const long w = (long)g.V * 12;   // float-float: one right-hand side at a time
    for (int y = 0; y < nrhs; y++)
        if (tol[y] > 0) ST(sign_ff(b + y * w, out + y * w, tol[y], mode));
    return OVL_OK;
}

// FP32 version for the inner (low-accuracy) D_N: b, out FP32 eo spinors.
ovl_status Ctx::sign32(const float4 *b, float4 *out, double tol, int mode, int store) {
    PhaseClock pclk(this, &t_sign_low);
    Ctx *c = this;
    int iters = 0, n = npole;
    const float4 *y;
    std::vector<double> dc;
    const float4 *b_orig = b;
    if (ndefl) {   // as in sign64: the multishift sees Pi b
        ST(defl_project32(b, defl_tmp32, dc));
        b = defl_tmp32;
    }
    if (store < 0) store = p.precision == OVL_MIXED_HALF ? 1 : p.precision == OVL_MIXED_BF16 ? 2 : 0;
    ovl_status ms = OVL_OK;
    if (store != 0) {
        // shifted directions stored in 16 bits (per site: 48 B, + 4 B norm for FP16, read and written)
        const bool bf = store == 2;
        ST(ensure_msh());
        ST(ms_setup(msh_state, tol, &n));
        CK(ms_init_half(g, n, msh_state, msh, b, rs, bf, stream));
        auto fn = [&](cudaEvent_t *e, unsigned f) {
            return ms_iter_half(g, U32, (float)m0_ker, msh_state, msh, rs, bf, stream, e, f);
        };
        ms = ms_run(msh_state, 1, bf ? 6 : 2, bf ? 96.0 : 104.0, false, fn, &iters);
        if (ms != OVL_OK && ms != OVL_ENOCONV) return ms;
        y = msh.y;
    } else {
        ST(ensure_ms32());
        ST(ms_setup(ms32_state, tol, &n));
        CK(ms_init_f32(g, n, ms32_state, ms32, b, rs, stream));
        auto fn = [&](cudaEvent_t *e, unsigned f) {
            return ms_iter_f32(g, U32, (float)m0_ker, ms32_state, ms32, rs, stream, e, f);
        };
        ms = ms_run(ms32_state, 1, 1, 48.0 * 4.0, g.tps32 != 4, fn, &iters);
        if (ms != OVL_OK && ms != OVL_ENOCONV) return ms;
        y = ms32.y;
    }
    stat_ms32 += iters;
    const float sc = (float)(zs_d0[n - 1] / lam_min);
    if (mode == 0) CK(wilson_f32(g, U32, y, out, (float)m0_ker, 1, sc, nullptr, 0.f, stream));
    else CK(wilson_f32(g, U32, y, out, (float)m0_ker, 0, sc, b_orig, (float)rho, stream));
    if (ndefl) ST(defl_add32(dc, out, mode));
    return ms;
}

ovl_status Ctx::ensure_ms64() {
    if (ms64.p) return OVL_OK;
    const long words = (long)g.V * 12;   // double2 per vector
    void *buf;
    ST(alloc(&buf, (size_t)words * sizeof(double2) * (npole + 3)));
    double2 *b2 = (double2 *)buf;
    ms64.r = b2;
    ms64.t = b2 + words;
    ms64.y = b2 + 2 * words;
    ms64.p = b2 + 3 * words;
    ms64.stride = words;
    return OVL_OK;
}
// ---- several right-hand sides
ovl_status Ctx::ensure_batch() {
    Ctx *c = this;
    if (msb_state) return OVL_OK;
    void *buf;
    ST(alloc(&buf, sizeof(MsState) * kMaxBatch));
    msb_state = (MsState *)buf;
    ST(alloc(&buf, sizeof(double) * (size_t)kMaxBatch * 2 * kMaxRedBlocks + 256));
    rsb.partials = (double *)buf;
    rsb.counter = (unsigned *)((char *)buf + sizeof(double) * (size_t)kMaxBatch * 2 * kMaxRedBlocks);
    ST(alloc(&buf, sizeof(unsigned) * kMaxBatch));
    bcounters = (unsigned *)buf;
    CK(cudaMemsetAsync(rsb.counter, 0, sizeof(unsigned), stream));
    CK(cudaMemsetAsync(bcounters, 0, sizeof(unsigned) * kMaxBatch, stream));
    CK(cudaMallocHost(&h_pinned_b, sizeof(MsState) * kMaxBatch + 4096));
    h_msb = (MsState *)h_pinned_b;
    h_msb_small = (int *)((char *)h_pinned_b + sizeof(MsState) * kMaxBatch);
    return OVL_OK;
}

// Lock-step multishift solves of nrhs right-hand sides (tolerance tol[y] each); the
// host polls the first four words (n, iter, done, status) of every state per chunk.
template <typename ST, typename Init, typename Iter>
ovl_status Ctx::msb_run(int nrhs, const double *tol, int n, int slot, Init init_fn, Iter iter_fn, long *iters_out) {
    Ctx *c = this;
    for (int y = 0; y < nrhs; y++) {
        MsState &s = h_msb[y];
        fill_poles(s, n, tol[y] > 0 ? tol[y] : 1.0);
        if (!(tol[y] > 0)) s.done = 1;   // a right-hand side that needs no work this time
    }
    CK(cudaMemcpyAsync(msb_state, h_msb, sizeof(MsState) * nrhs, cudaMemcpyHostToDevice, stream));
    CK(init_fn());
    const int chunk = std::min(p.check_every, kMaxChunk);
    GraphSlot &gs = graphs[slot];
    if (gs.exec && (gs.nrhs != nrhs || gs.chunk != chunk)) {
        cudaGraphExecDestroy(gs.exec);
        gs.exec = nullptr;
    }
    int done_iters = 0;
    while (true) {
        if (p.use_graphs) {
            if (!gs.exec) {
                cudaGraph_t graph;
                set_launch_counting(false);
                CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t ce = cudaSuccess;
                for (int k = 0; k < chunk && ce == cudaSuccess; k++) ce = iter_fn();
                cudaError_t ee = cudaStreamEndCapture(stream, &graph);
                set_launch_counting(true);
                CK(ce);
                CK(ee);
                cudaError_t ie = cudaGraphInstantiate(&gs.exec, graph, 0);
                cudaGraphDestroy(graph);
                CK(ie);
                gs.nrhs = nrhs;
                gs.chunk = chunk;
            }
            CK(cudaGraphLaunch(gs.exec, stream));
            count_launches(3L * chunk);
        } else {
            for (int k = 0; k < chunk; k++) CK(iter_fn());
        }
        done_iters += chunk;
        CK(cudaMemcpy2DAsync(h_msb_small, 4 * sizeof(int), msb_state, sizeof(MsState), 4 * sizeof(int), nrhs,
                             cudaMemcpyDeviceToHost, stream));
        ST(sync());
        bool all = true;
        long itmax = 0;
        for (int y = 0; y < nrhs; y++) {
            const int *h = h_msb_small + 4 * y;
            if (h[3]) {
                err = "batched multishift CG breakdown (non-finite or non-positive scalar)";
                return OVL_EBREAKDOWN;
            }
            all = all && h[2];
            itmax = std::max(itmax, (long)h[1]);
        }
        if (!all && past_deadline()) return OVL_ETIMEOUT;
        if (all) {
            *iters_out = itmax;
            return OVL_OK;
        }
        if (itmax >= p.max_ms_iter || done_iters > p.max_ms_iter + chunk) {
            *iters_out = itmax;
            err = "batched multishift CG reached max_ms_iter";
            return OVL_ENOCONV;
        }
    }
}

// Smallest positive tolerance of a batch (the most demanding right-hand side sets the
// Zolotarev degree of the whole batch); 1 if none is positive.
static double min_positive(const double *tol, int n) {
    double m = 1.0;
    for (int y = 0; y < n; y++)
        if (tol[y] > 0 && tol[y] < m) m = tol[y];
    return m;
}

ovl_status Ctx::sign64_batch(const double2 *b, double2 *out, int nrhs, const double *tol, int mode) {
    Ctx *c = this;
    if (ndefl || p.sign_method == OVL_SIGN_KRYLOV) {   // deflation and the Krylov sign run one at a time
        const long w = (long)g.V * 12;
        for (int y = 0; y < nrhs; y++)
            if (tol[y] > 0) ST(sign64(b + y * w, out + y * w, tol[y], mode));
        return OVL_OK;
    }
    ST(ensure_batch());
    if (!msb64.p || msb64_cap < nrhs) {   // sized to the batch (grown when a larger one comes)
        if (msb64.p) {
            cudaFree(msb64.r);
            allocs.erase(std::find(allocs.begin(), allocs.end(), (void *)msb64.r));
        }
        const long words = (long)g.V * 12;
        void *buf;
        ST(alloc(&buf, (size_t)words * sizeof(double2) * nrhs * (npole + 3)));
        double2 *d = (double2 *)buf;
        msb64.r = d;
        msb64.t = d + words * nrhs;
        msb64.y = d + 2 * words * nrhs;
        msb64.p = d + 3 * words * nrhs;
        msb64.stride = words;
        msb64_cap = nrhs;
    }
    long iters = 0;
    auto init = [&]() { return msb_init_f64(g, nrhs, npole, msb_state, msb64, b, rsb, stream); };
    auto it = [&]() { return msb_iter_f64(g, U64, m0_ker, nrhs, npole, msb_state, msb64, rsb, bcounters, stream); };
    const int n = pick_poles(min_positive(tol, nrhs));
    ST((msb_run<double2>(nrhs, tol, n, 3, init, it, &iters)));
    stat_ms64 += iters * nrhs;
    const double sc = zs_d0[n - 1] / lam_min;
    CK(wilson_batch_f64(g, U64, msb64.y, out, msb64.stride, nrhs, m0_ker, mode == 0, sc, mode == 1 ? b : nullptr,
                        rho, stream));
    return OVL_OK;
}

ovl_status Ctx::sign32_batch(const float4 *b, float4 *out, int nrhs, const double *tol, int mode) {
    Ctx *c = this;
    if (ndefl) {
        const long w = (long)g.V * 6;
        for (int y = 0; y < nrhs; y++)
            if (tol[y] > 0) ST(sign32(b + y * w, out + y * w, tol[y], mode));
        return OVL_OK;
    }
    ST(ensure_batch());
    if (!msb32.p || msb32_cap < nrhs) {
        if (msb32.p) {
            cudaFree(msb32.r);
            allocs.erase(std::find(allocs.begin(), allocs.end(), (void *)msb32.r));
        }
        const long words = (long)g.V * 6;
        void *buf;
        ST(alloc(&buf, (size_t)words * sizeof(float4) * nrhs * (npole + 3)));
        float4 *d = (float4 *)buf;
        msb32.r = d;
        msb32.t = d + words * nrhs;
        msb32.y = d + 2 * words * nrhs;
        msb32.p = d + 3 * words * nrhs;
        msb32.stride = words;
        msb32_cap = nrhs;
    }
    long iters = 0;
    auto init = [&]() { return msb_init_f32(g, nrhs, npole, msb_state, msb32, b, rsb, stream); };
    auto it = [&]() {
        return msb_iter_f32(g, U32, (float)m0_ker, nrhs, npole, msb_state, msb32, rsb, bcounters, stream);
    };
    const int n = pick_poles(min_positive(tol, nrhs));
    ST((msb_run<float4>(nrhs, tol, n, 4, init, it, &iters)));
    stat_ms32 += iters * nrhs;
    const float sc = (float)(zs_d0[n - 1] / lam_min);
    CK(wilson_batch_f32(g, U32, msb32.y, out, msb32.stride, nrhs, (float)m0_ker, mode == 0, sc,
                        mode == 1 ? b : nullptr, (float)rho, stream));
    return OVL_OK;
}

ovl_status Ctx::ensure_msh() {
    if (msh.ph) return OVL_OK;
    if (!msh_state) {
        void *sb;
        ST(alloc(&sb, sizeof(MsState)));
        msh_state = (MsState *)sb;
    }
    const long words = (long)g.V * 6, words_h = (long)g.V * 3;
    const int nh = npole > 1 ? npole - 1 : 1;
    void *buf;
    ST(alloc(&buf, (size_t)words * sizeof(float4) * 4 + (size_t)words_h * sizeof(uint4) * nh +
                       (size_t)g.V * sizeof(float) * nh));
    float4 *f = (float4 *)buf;
    msh.r = f;
    msh.t = f + words;
    msh.y = f + 2 * words;
    msh.p0 = f + 3 * words;
    msh.ph = (uint4 *)(f + 4 * words);
    msh.pn = (float *)(msh.ph + (size_t)words_h * nh);
    msh.words = words;
    msh.words_h = words_h;
    return OVL_OK;
}

ovl_status Ctx::ensure_ms32() {
    if (ms32.p) return OVL_OK;
    const long words = (long)g.V * 6;    // float4 per vector
    void *buf;
    ST(alloc(&buf, (size_t)words * sizeof(float4) * (npole + 4)));
    float4 *b4 = (float4 *)buf;
    ms32.r = b4;
    ms32.t = b4 + words;
    ms32.y = b4 + 2 * words;
    ms32.p = b4 + 3 * words;
    ms32.r2 = b4 + (3 + npole) * words;
    ms32.stride = words;
    return OVL_OK;
}

// ------------------------------------------------------------------ spectral estimates
// Tridiagonal eigenvalue bounds by Sturm-sequence bisection.
static int sturm_count(const std::vector<double> &a, const std::vector<double> &b, int m, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; i++) {
        const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0) cnt++;
    }
    return cnt;
}
static double tridiag_eig(const std::vector<double> &a, const std::vector<double> &b, int m, int k) {
    // k-th smallest eigenvalue (0-based) of the m x m symmetric tridiagonal (a, b)
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; i++) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(fabs(lo), fabs(hi)); it++) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, m, mid) > k) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Lanczos on Q^2 in FP32 (no re-orthogonalisation: extremal Ritz values converge
// first and spurious copies do not move them).
ovl_status Ctx::lanczos_bounds(double *lmin, double *lmax, double m0) {
    Ctx *c = this;
    const float mq = (float)(isnan(m0) ? m0_ker : m0);   // Q = Gamma5 D_W(mq)
    const long nf = n64;   // floats per FP32 vector
    float *v0, *v1, *w, *tt;
    void *buf;
    ST(alloc(&buf, (size_t)nf * sizeof(float) * 4));
    v0 = (float *)buf;
    v1 = v0 + nf;
    w = v1 + nf;
    tt = w + nf;
    // deterministic start vector
    std::vector<float> h(nf);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (long i = 0; i < nf; i++) {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        h[i] = (float)((double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
    CK(cudaMemcpyAsync(v1, h.data(), nf * sizeof(float), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(v0, 0, nf * sizeof(float), stream));
    double nn;
    ST(norm2_f(v1, &nn));
    CK(dev_axpby_f((float)(1.0 / sqrt(nn)), v1, 0.f, v1, nf, stream));
    std::vector<double> al, be;
    double prev_min = 0, prev_max = 0, tmin = 0, tmax = 0;
    const int maxit = 600;
    double beta_prev = 0.0;
    for (int j = 0; j < maxit; j++) {
        CK(wilson_f32(g, U32, (const float4 *)v1, (float4 *)tt, mq, 1, 1.f, nullptr, 0.f, stream));
        CK(wilson_f32(g, U32, (const float4 *)tt, (float4 *)w, mq, 1, 1.f, nullptr, 0.f, stream));
        if (j > 0) CK(dev_axpby_f((float)(-beta_prev), v0, 1.f, w, nf, stream));
        double d2[2];
        CK(dev_cdot_f(v1, w, nf, d_scal, rs, stream));
        ST(fetch(d_scal, 2, d2));
        const double alpha = d2[0];
        CK(dev_axpby_f((float)(-alpha), v1, 1.f, w, nf, stream));
        double bb;
        ST(norm2_f(w, &bb));
        const double beta = sqrt(bb);
        al.push_back(alpha);
        be.push_back(beta);
        const int m = j + 1;
        if (m % 10 == 0 || beta == 0.0) {
            tmin = tridiag_eig(al, be, m, 0);
            tmax = tridiag_eig(al, be, m, m - 1);
            if (m >= 30 && fabs(tmin - prev_min) <= 1e-4 * tmin && fabs(tmax - prev_max) <= 1e-5 * tmax) break;
            prev_min = tmin;
            prev_max = tmax;
        }
        if (beta == 0.0) break;
        // v0 <- v1, v1 <- w / beta
        CK(cudaMemcpyAsync(v0, v1, nf * sizeof(float), cudaMemcpyDeviceToDevice, stream));
        CK(dev_axpby_f((float)(1.0 / beta), w, 0.f, v1, nf, stream));
        beta_prev = beta;
    }
    if (!(tmin > 0) || !(tmax > tmin)) {
        err = "Lanczos could not bound the spectrum of Q^2 (Q singular?)";
        return OVL_EINVAL;
    }
    *lmin = sqrt(tmin);
    *lmax = sqrt(tmax);
    return OVL_OK;
}

// sigma_min of Eq. (default_m): the smallest real part of the eigenvalues of D_W(0). It is
// estimated by the smallest singular value of D_W(0), i.e. the smallest |eigenvalue| of the
// Hermitian Q(0) = Gamma5 D_W(0), from the Lanczos run on Q(0)^2 (its extreme eigenvalues
// converge fast and no basis is stored). For the near-real low modes of smeared fields the two
// quantities are close. (Sec. 5.1's power-iteration guess 8 - sigma_max, rounded up, only
// bounds the range of the paper's m0_prec scan; taken as sigma_min it put m0_prec near the
// critical mass and made the Wilson solves much slower.)
ovl_status Ctx::sigma_min_estimate(double *smin) {
    double lo, hi;
    ST(lanczos_bounds(&lo, &hi, 0.0));
    *smin = lo;
    return OVL_OK;
}

// ------------------------------------------------------------------ autotuner
// Threads per site of the stencils (1 or 4) for this lattice shape: both variants of
// each precision are timed with CUDA events on the context's stream and the faster is
// kept. Results are cached per process and shape.
static std::mutex g_tune_mu;
struct TuneEntry {
    int tps64, tps32;
    float ms[4];
};
static std::map<std::tuple<int, int, int, int>, TuneEntry> g_tune_cache;

ovl_status Ctx::autotune() {
    Ctx *c = this;
    const auto key = std::make_tuple(g.L[0], g.L[1], g.L[2], g.L[3]);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            g.tps64 = it->second.tps64;
            g.tps32 = it->second.tps32;
            for (int k = 0; k < 4; k++) tune_ms[k] = it->second.ms[k];
            return OVL_OK;
        }
    }
    void *buf;
    ST(alloc(&buf, (size_t)n64 * sizeof(float) * 2));
    float4 *fa = (float4 *)buf, *fb = fa + (size_t)g.V * 6;
    CK(cudaMemsetAsync(buf, 0, (size_t)n64 * sizeof(float) * 2, stream));
    CK(cudaMemsetAsync(io_a, 0, (size_t)n64 * sizeof(double), stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = g.V >= (1 << 20) ? 5 : 20;
    float best[2][2];
    for (int prec = 0; prec < 2; prec++) {
        for (int v = 0; v < 2; v++) {
            const int tps = v == 0 ? 1 : 4;
            Geom gg = g;
            gg.tps64 = gg.tps32 = tps;
            for (int k = 0; k < 3 + reps; k++) {
                if (k == 3) CK(cudaEventRecord(e0, stream));
                if (prec == 0) CK(wilson_f64(gg, U64, io_a, io_b, m0_ker, 0, 1.0, nullptr, 0.0, stream));
                else CK(wilson_f32(gg, U32, fa, fb, (float)m0_ker, 0, 1.f, nullptr, 0.f, stream));
            }
            CK(cudaEventRecord(e1, stream));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&best[prec][v], e0, e1));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g.tps64 = best[0][1] < best[0][0] ? 4 : 1;
    g.tps32 = best[1][1] < best[1][0] ? 4 : 1;
    tune_ms[0] = best[0][0] / reps;
    tune_ms[1] = best[0][1] / reps;
    tune_ms[2] = best[1][0] / reps;
    tune_ms[3] = best[1][1] / reps;
    {
        // first writer wins: a context of the same shape that finished tuning first (for
        // instance concurrently in the serving loop) has fixed the variant for the whole
        // process, so that every context of one lattice shape runs the same kernels and
        // gets bit-identical results whatever else is running
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            g.tps64 = it->second.tps64;
            g.tps32 = it->second.tps32;
            for (int k = 0; k < 4; k++) tune_ms[k] = it->second.ms[k];
        } else {
            g_tune_cache[key] = TuneEntry{g.tps64, g.tps32, {tune_ms[0], tune_ms[1], tune_ms[2], tune_ms[3]}};
        }
    }
    cudaFree(buf);
    allocs.erase(std::find(allocs.begin(), allocs.end(), buf));
    return OVL_OK;
}

// FP32 multi-RHS stencil kernels (Geom::mrhs32 for blocks of up to 6 right-hand sides,
// mrhs32l for 7..12): each of the three kernels is timed on 4 and on 12 right-hand sides of
// seeded pseudo-random fields and the fastest per right-hand side kept for each block size
// (their order changes with the block: at 64x32^3 the 32-site tiles are the fastest at 4 and
// the slowest at 12). Cached per process and lattice shape; the first context of a shape to
// finish fixes the choice (as for the threads per site), so every context of that shape runs
// the same kernels.
static std::map<std::tuple<int, int, int, int>, std::pair<std::array<int, 2>, std::array<float, 6>>> g_mrhs_cache;
ovl_status Ctx::autotune_mrhs() {
    Ctx *c = this;
    const auto key = std::make_tuple(g.L[0], g.L[1], g.L[2], g.L[3]);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_mrhs_cache.find(key);
        if (it != g_mrhs_cache.end()) {
            g.mrhs32 = it->second.first[0];
            g.mrhs32l = it->second.first[1];
            for (int k = 0; k < 6; k++) tune_mrhs_ms[k] = it->second.second[k];
            return OVL_OK;
        }
    }
    constexpr int nmax = 12;
    const long w = (long)g.V * 6;   // float4 words per FP32 vector
    void *buf;
    ST(alloc(&buf, (size_t)w * 2 * nmax * sizeof(float4)));
    float4 *fin = (float4 *)buf, *fout = fin + w * nmax;
    CK(fill_random_f32((float *)fin, 4 * w * nmax, 7301, stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = g.V >= (1 << 20) ? 3 : 10;
    float ms[6] = {0, 0, 0, 0, 0, 0};
    int best[2] = {0, 0};
    for (int sz = 0; sz < 2; sz++) {
        const int nr = sz ? nmax : 4;
        for (int v = 0; v < 3; v++) {
            Geom gg = g;
            gg.mrhs32 = gg.mrhs32l = v + 1;
            for (int k = 0; k < 2 + reps; k++) {
                if (k == 2) CK(cudaEventRecord(e0, stream));
                CK(wilson_batch_f32(gg, U32, fin, fout, w, nr, (float)m0_ker, 0, 1.f, nullptr, 0.f, stream));
            }
            CK(cudaEventRecord(e1, stream));
            CK(cudaEventSynchronize(e1));
            float t = 0;
            CK(cudaEventElapsedTime(&t, e0, e1));
            ms[3 * sz + v] = t / (float)(reps * nr);
            if (ms[3 * sz + v] < ms[3 * sz + best[sz]]) best[sz] = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g.mrhs32 = best[0] + 1;
    g.mrhs32l = best[1] + 1;
    for (int k = 0; k < 6; k++) tune_mrhs_ms[k] = ms[k];
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_mrhs_cache.find(key);
        if (it != g_mrhs_cache.end()) {
            g.mrhs32 = it->second.first[0];
            g.mrhs32l = it->second.first[1];
            for (int k = 0; k < 6; k++) tune_mrhs_ms[k] = it->second.second[k];
        } else {
            g_mrhs_cache[key] = {{g.mrhs32, g.mrhs32l}, {ms[0], ms[1], ms[2], ms[3], ms[4], ms[5]}};
        }
    }
    cudaFree(buf);
    allocs.erase(std::find(allocs.begin(), allocs.end(), buf));
    return OVL_OK;
}

// Threads per site of the FP32 Schwarz block kernel (1, 2 or 4): one Schwarz cycle of
// each variant is timed on a constant non-zero input and the fastest kept. Cached per
// process, lattice shape and block shape.
static std::map<std::tuple<int, int, int, int, int, int, int, int, int>, std::pair<int, std::array<float, 3>>>
    g_sap_cache;

ovl_status Ctx::autotune_sap() {
    Ctx *c = this;
    const auto key = std::make_tuple(g.L[0], g.L[1], g.L[2], g.L[3], p.sap_block[0], p.sap_block[1], p.sap_block[2],
                                     p.sap_block[3], p.sap_mr_iters);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_sap_cache.find(key);
        if (it != g_sap_cache.end()) {
            sap_tps = it->second.first;
            for (int k = 0; k < 3; k++) sap_ms[k] = it->second.second[k];
            return OVL_OK;
        }
    }
    void *buf;
    const size_t bytes = (size_t)n64 * sizeof(float);
    ST(alloc(&buf, bytes * 3));
    float4 *fv = (float4 *)buf, *fx = (float4 *)((char *)buf + bytes), *fr = (float4 *)((char *)buf + 2 * bytes);
    CK(cudaMemsetAsync(fv, 0x3c, bytes, stream));   // every float 0x3c3c3c3c ~ 0.0115
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = g.V >= (1 << 20) ? 3 : 10;
    const int tps_of[3] = {1, 2, 4};
    float best = 0.f;
    int best_tps = 1;
    for (int v = 0; v < 3; v++) {
        SapGeom sg = make_sap_geom(g, p.sap_block);
        sg.tps = tps_of[v];
        for (int k = 0; k < 2 + reps; k++) {
            if (k == 2) CK(cudaEventRecord(e0, stream));
            CK(sap_f32(g, sg, U32, fv, fx, fr, -0.5f, 1, p.sap_mr_iters, stream));
        }
        CK(cudaEventRecord(e1, stream));
        CK(cudaEventSynchronize(e1));
        float ms;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        sap_ms[v] = ms / reps;
        if (v == 0 || sap_ms[v] < best) {
            best = sap_ms[v];
            best_tps = tps_of[v];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sap_tps = best_tps;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);   // first writer wins, as in autotune()
        auto it = g_sap_cache.find(key);
        if (it != g_sap_cache.end()) {
            sap_tps = it->second.first;
            for (int k = 0; k < 3; k++) sap_ms[k] = it->second.second[k];
        } else {
            g_sap_cache[key] = {sap_tps, {sap_ms[0], sap_ms[1], sap_ms[2]}};
        }
    }
    cudaFree(buf);
    allocs.erase(std::find(allocs.begin(), allocs.end(), buf));
    return OVL_OK;
}

// ------------------------------------------------------------------ ABI
extern "C" ovl_status ovl_zolotarev(double k, int n, double *d0, double *a, double *c, double *delta) {
    if (!d0 || !a || !c || !delta) return OVL_EINVAL;
    return zolotarev_host(k, n, d0, a, c, delta) == 0 ? OVL_OK : OVL_EINVAL;
}

ovl_status Ctx::set_zolotarev() {
    const double k = lam_min / lam_max;
    za.assign(npole, 0.0);
    zc.assign(npole, 0.0);
    if (zolotarev_host(k, npole, &zd0, za.data(), zc.data(), &zdelta) != 0) {
        err = "Zolotarev coefficients: bad interval";
        return OVL_EINVAL;
    }
    zs_d0.assign(npole, 0.0);
    zs_delta.assign(npole, 0.0);
    zs_a.assign(npole, std::vector<double>());
    zs_c.assign(npole, std::vector<double>());
    for (int n = 1; n <= npole; n++) {
        zs_a[n - 1].assign(n, 0.0);
        zs_c[n - 1].assign(n, 0.0);
        if (zolotarev_host(k, n, &zs_d0[n - 1], zs_a[n - 1].data(), zs_c[n - 1].data(), &zs_delta[n - 1]) != 0) {
            err = "Zolotarev coefficients: bad interval";
            return OVL_EINVAL;
        }
    }
    return OVL_OK;
}

static ovl_status create_impl(Ctx *c, const double *gauge, const int dims[4], double rho_in, double mu,
                              const ovl_params *pp, void *stream) {
    if (pp) c->p = *pp;
    else ovl_params_default(&c->p);
    for (int m = 0; m < 4; m++) {
        if (dims[m] < 2 || (dims[m] & 1)) {
            c->err = "lattice extents must be even and >= 2";
            return OVL_EINVAL;
        }
    }
    ST(validate_params(c->p, dims, c->err));
    if (!(mu > 0) || !(rho_in > 0) || !(mu < 2 * rho_in)) {
        c->err = "need rho > 0 and 0 < mu < 2 rho";
        return OVL_EINVAL;
    }
    long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (1L << 26)) {
        c->err = "lattice too large";
        return OVL_EINVAL;
    }
    for (int m = 0; m < 4; m++) c->g.L[m] = dims[m];
    c->g.V = (int)V;
    c->g.Vh = (int)(V / 2);
    c->g.Lh3 = dims[3] / 2;
    c->g.antiperiodic = c->p.antiperiodic;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess) {
            cudaGetLastError();
            c->err = "no usable CUDA device";
            return OVL_ECUDA;
        }
        c->g.nsm = nsm;
    }
    c->n64 = V * 24;
    c->m0_ker = -rho_in;
    c->rho_in = rho_in;
    c->mu = mu;
    c->rho = (-mu / 2.0 + c->m0_ker) / (mu / 2.0 + c->m0_ker);   // Sec. 5
    c->npole = c->p.n_poles;
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    // pinned host scratch: scalars, flags, multishift state copies
    CK(cudaMallocHost(&c->h_pinned, (size_t)kScal * sizeof(double) + (1 << 16)));
    c->h_scal = (double *)c->h_pinned;
    char *hp = (char *)c->h_pinned + (size_t)kScal * sizeof(double);
    c->h_flag = (int *)hp;
    c->h_ms_small = (int *)(hp + 4096);
    c->h_ms = (MsState *)(hp + 8192);
    c->h_hist = (int *)(hp + 32768);
    c->launch_mark = launches_total();
    // device scratch
    void *buf;
    ST(c->alloc(&buf, sizeof(double) * kMaxRedValues * kMaxRedBlocks + 4096));
    c->rs.partials = (double *)buf;
    c->rs.counter = (unsigned *)((char *)buf + sizeof(double) * kMaxRedValues * kMaxRedBlocks);
    c->d_flag = (int *)((char *)buf + sizeof(double) * kMaxRedValues * kMaxRedBlocks + 256);
    CK(cudaMemsetAsync(buf, 0, sizeof(double) * kMaxRedValues * kMaxRedBlocks + 4096, c->stream));
    ST(c->alloc(&buf, (size_t)kScal * sizeof(double)));
    c->d_scal = (double *)buf;
    ST(c->alloc(&buf, sizeof(MsState)));
    c->ms64_state = (MsState *)buf;
    ST(c->alloc(&buf, sizeof(MsState)));
    c->ms32_state = (MsState *)buf;
    ST(c->alloc(&buf, (size_t)128 * 256 * 2 * sizeof(double)));
    c->d_md_part = (double *)buf;
    ST(c->alloc(&buf, (size_t)2 * 128 * sizeof(double)));
    c->d_coef = (double *)buf;
    // gauge field
    ST(c->alloc((void **)&c->U64, (size_t)V * 4 * kLink64Words * sizeof(double2)));
    ST(c->alloc((void **)&c->U32, (size_t)V * 4 * 3 * sizeof(float4)));
    ST(c->alloc((void **)&c->io_lex, (size_t)c->n64 * sizeof(double)));
    ST(c->alloc((void **)&c->io_a, (size_t)c->n64 * sizeof(double)));
    ST(c->alloc((void **)&c->io_b, (size_t)c->n64 * sizeof(double)));
    const double *glex = gauge;
    void *gtmp = nullptr;
    if (!is_device_ptr(gauge)) {
        const size_t gb = (size_t)V * 4 * 9 * 2 * sizeof(double);
        ST(c->alloc(&gtmp, gb));
        CK(cudaMemcpyAsync(gtmp, gauge, gb, cudaMemcpyHostToDevice, c->stream));
        glex = (const double *)gtmp;
    }
    CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    CK(pack_gauge(c->g, glex, c->U64, c->U32, c->d_flag, 1e-10, c->stream));
    CK(cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ST(c->sync());
    if (gtmp) {
        cudaFree(gtmp);
        c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), gtmp));
    }
    if (*c->h_flag) {
        c->err = "gauge field: some link is not SU(3) to 1e-10 (or holds NaN)";
        return OVL_EINVAL;
    }
    c->g.tps64 = c->g.tps32 = 1;
    if (c->p.stencil_tps) c->g.tps64 = c->g.tps32 = c->p.stencil_tps;
    else ST(c->autotune());
    if (c->p.mrhs_kernel) c->g.mrhs32 = c->g.mrhs32l = c->p.mrhs_kernel;
    else ST(c->autotune_mrhs());
    if (c->p.sap_tps) {
        c->sap_tps = c->p.sap_tps;
        c->sap_tuned = true;
    } else if (c->p.precond != OVL_PREC_NONE) {
        ST(c->autotune_sap());
        c->sap_tuned = true;
    }
    // spectral interval of |Q|
    if (c->p.lambda_min > 0) {
        c->lam_min = c->p.lambda_min;
        c->lam_max = c->p.lambda_max;
        c->lam_estimated = false;
    } else {
        double lmin, lmax;
        ST(c->lanczos_bounds(&lmin, &lmax));
        c->lam_min = 0.9 * lmin;    // margins: Ritz values bound the extreme eigenvalues from inside
        c->lam_max = 1.05 * lmax;
        c->lam_estimated = true;
    }
    if (c->p.n_deflate > 0) {   // the rational approximation then starts at 0.9 |lambda_{k+1}|
        ST(c->deflation_setup());
        c->lam_min = std::max(c->lam_min, 0.9 * c->defl_next);
    }
    ST(c->set_zolotarev());
    // preconditioner mass m0^def (Eq. default_m) unless given
    c->sigma_min = NAN;
    if (isnan(c->p.m0_prec) && c->p.precond != OVL_PREC_NONE) {
        ST(c->sigma_min_estimate(&c->sigma_min));
        c->m0_prec = (-c->m0_ker - c->sigma_min) * c->rho + c->m0_ker;
    } else {
        c->m0_prec = c->p.m0_prec;
    }
    return OVL_OK;
}

extern "C" ovl_status ovl_create(ovl_ctx **ctx, const double *gauge, const int dims[4], double rho_in, double mu,
                                 const ovl_params *p, void *cuda_stream) {
    if (!ctx) return OVL_EINVAL;
    *ctx = nullptr;
    if (!gauge || !dims) {
        g_create_error = "ovl_create: NULL gauge or dims";
        return OVL_EINVAL;
    }
    Ctx *c = new Ctx();
    ovl_status s = create_impl(c, gauge, dims, rho_in, mu, p, cuda_stream);
    if (s != OVL_OK) {
        g_create_error = c->err;
        delete c;
        return s;
    }
    *ctx = reinterpret_cast<ovl_ctx *>(c);
    return OVL_OK;
}

extern "C" ovl_status ovl_destroy(ovl_ctx *ctx) {
    delete reinterpret_cast<Ctx *>(ctx);
    return OVL_OK;
}

extern "C" const char *ovl_last_error(const ovl_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return reinterpret_cast<const Ctx *>(ctx)->err.c_str();
}

extern "C" ovl_status ovl_info(const ovl_ctx *ctx, double *lambda_min, double *lambda_max, double *delta, double *rho,
                               double *m0_ker, double *m0_prec, double *sigma_min) {
    if (!ctx) return OVL_EINVAL;
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (lambda_min) *lambda_min = c->lam_min;
    if (lambda_max) *lambda_max = c->lam_max;
    if (delta) *delta = c->zdelta;
    if (rho) *rho = c->rho;
    if (m0_ker) *m0_ker = c->m0_ker;
    if (m0_prec) *m0_prec = c->m0_prec;
    if (sigma_min) *sigma_min = c->sigma_min;
    return OVL_OK;
}

static ovl_status check_ctx_ptrs(Ctx *c, const void *a, const void *b) {
    if (!c) return OVL_EINVAL;
    if (!a || !b) {
        c->err = "NULL vector argument";
        return OVL_EINVAL;
    }
    return OVL_OK;
}

extern "C" ovl_status wilson_apply(ovl_ctx *ctx, double *out, const double *in, double m0) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    if (!isfinite(m0)) {
        c->err = "m0 must be finite";
        return OVL_EINVAL;
    }
    ST(c->import_vec(in, c->io_a));
    CK(wilson_f64(c->g, c->U64, c->io_a, c->io_b, m0, 0, 1.0, nullptr, 0.0, c->stream));
    return c->export_vec(c->io_b, out);
}

static ovl_status check_tol(Ctx *c, double tol) {
    if (!(tol >= 1e-14 && tol < 1.0)) {
        c->err = "tol must be in [1e-14, 1)";
        return OVL_EINVAL;
    }
    return OVL_OK;
}

extern "C" ovl_status sign_apply(ovl_ctx *ctx, double *out, const double *in, double tol) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    ST(check_tol(c, tol));
    ST(c->import_vec(in, c->io_a));
    const ovl_status st = c->sign64(c->io_a, c->io_b, tol, 0);
    if (st != OVL_OK && st != OVL_ENOCONV) return st;
    ST(c->export_vec(c->io_b, out));
    return st;
}

extern "C" ovl_status ovl_apply(ovl_ctx *ctx, double *out, const double *in, double tol) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    ST(check_tol(c, tol));
    ST(c->import_vec(in, c->io_a));
    const ovl_status st = c->sign64(c->io_a, c->io_b, tol, 1);
    if (st != OVL_OK && st != OVL_ENOCONV) return st;
    ST(c->export_vec(c->io_b, out));
    return st;
}

extern "C" ovl_status ovl_solve(ovl_ctx *ctx, double *x, const double *b, int n_rhs, double tol, ovl_stats *stats) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, x, b));
    if (n_rhs < 1) {
        c->err = "n_rhs must be >= 1";
        return OVL_EINVAL;
    }
    if (tol == 0.0) tol = c->p.tol_outer;
    ST(check_tol(c, tol));
    return solve_all(c, x, b, n_rhs, tol, stats);
}

extern "C" ovl_status ovl_prof_enable(ovl_ctx *ctx, int on) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (on && !c->d_hist) {
        c->hist_cap = c->p.max_ms_iter + kMaxChunk;
        ST(c->alloc((void **)&c->d_hist, (size_t)c->hist_cap * sizeof(int)));
    }
    c->prof = on != 0;
    return OVL_OK;
}

extern "C" ovl_status ovl_prof_get(ovl_ctx *ctx, ovl_prof *out, int reset) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !out) return OVL_EINVAL;
    memset(out, 0, sizeof(*out));
    out->launches = launches_total() - c->launch_mark;
    out->valid = 1;
    const double V = (double)c->g.V;
    for (int w = 0; w < 3; w++) {
        const ProfAcc &pa = c->pacc[w];
        ovl_prof_kernel &st = out->k[2 * w], &sh = out->k[2 * w + 1];
        st.ms = pa.q_ms + pa.r_ms;
        st.timed = pa.q_t + pa.r_t;
        st.launches = 2 * pa.n;
        st.bytes = pa.q_bytes + pa.r_bytes;
        st.timed_bytes = pa.q_tb + pa.r_tb;
        st.flops = 1368.0 * V * (double)st.launches;
        sh.ms = pa.s_ms;
        sh.timed = pa.s_t;
        sh.launches = pa.n;
        sh.bytes = pa.s_bytes;
        sh.timed_bytes = pa.s_tb;
        if (!pa.valid) out->valid = 0;
    }
    if (reset) {
        for (int w = 0; w < 3; w++) c->pacc[w] = ProfAcc();
        c->launch_mark = launches_total();
    }
    return OVL_OK;
}

extern "C" ovl_status ovl_tuning(const ovl_ctx *ctx, int *tps64, int *tps32, float *ms) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (tps64) *tps64 = c->g.tps64;
    if (tps32) *tps32 = c->g.tps32;
    if (ms)
        for (int k = 0; k < 4; k++) ms[k] = c->tune_ms[k];
    return OVL_OK;
}

extern "C" ovl_status ovl_tuning_mrhs(const ovl_ctx *ctx, int *kernel, float *ms) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (kernel) {
        kernel[0] = c->g.mrhs32;
        kernel[1] = c->g.mrhs32l;
    }
    if (ms)
        for (int k = 0; k < 6; k++) ms[k] = c->tune_mrhs_ms[k];
    return OVL_OK;
}

extern "C" ovl_status ovl_hermitian_eig(int n, const double *A, double *w, double *Z) {
    if (n < 1 || !A || !w || !Z) return OVL_EINVAL;
    std::vector<std::complex<double>> a((size_t)n * n);
    for (size_t k = 0; k < (size_t)n * n; k++) a[k] = std::complex<double>(A[2 * k], A[2 * k + 1]);
    const int r = hermitian_eig(n, a.data(), w, reinterpret_cast<std::complex<double> *>(Z));
    return r == 0 ? OVL_OK : OVL_ENOCONV;
}

extern "C" ovl_status ovl_deflation_info(const ovl_ctx *ctx, int *k, double *lambda, double *lambda_next,
                                         double *setup_s, double *resid_max, long *matvecs) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (k) *k = c->ndefl;
    if (lambda)
        for (int i = 0; i < c->ndefl; i++) lambda[i] = c->defl_lambda[i];
    if (lambda_next) *lambda_next = c->defl_next;
    if (setup_s) *setup_s = c->defl_setup_s;
    if (resid_max) *resid_max = c->defl_resid;
    if (matvecs) *matvecs = c->defl_matvecs;
    return OVL_OK;
}

extern "C" ovl_status ovl_krylov_sign_info(const ovl_ctx *ctx, long *cycles, long *matvecs) {
    if (!ctx) return OVL_EINVAL;
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (cycles) *cycles = c->ks_cycles;
    if (matvecs) *matvecs = c->ks_matvecs;
    return OVL_OK;
}

extern "C" ovl_status ovl_m0_adapt_info(const ovl_ctx *ctx, double *cand, double *eff, long *uses, double *best) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    const Ctx::M0Adapt &a = c->m0a;
    double b = NAN, be = 0.0;
    for (int k = 0; k < 5; k++) {
        const bool have = k < (int)a.cand.size();
        const double e = have && a.cost[k] > 0 ? a.gain[k] / a.cost[k] : 0.0;
        if (cand) cand[k] = have ? a.cand[k] : 0.0;
        if (eff) eff[k] = e;
        if (have && e > be) {
            be = e;
            b = a.cand[k];
        }
    }
    if (uses) *uses = a.uses;
    if (best) *best = b;
    return OVL_OK;
}

extern "C" ovl_status ovl_tuning_sap(const ovl_ctx *ctx, int *tps, float *ms) {
    const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
    if (!c) return OVL_EINVAL;
    if (tps) *tps = c->sap_tps;
    if (ms)
        for (int k = 0; k < 3; k++) ms[k] = c->sap_ms[k];
    return OVL_OK;
}

extern "C" ovl_status wilson_solve(ovl_ctx *ctx, double *x, const double *b, double m0, double tol, int *iters) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, x, b));
    if (!isfinite(m0)) {
        c->err = "m0 must be finite";
        return OVL_EINVAL;
    }
    if (!(tol > 0 && tol < 1)) {
        c->err = "tol must be in (0, 1)";
        return OVL_EINVAL;
    }
    for (int m = 0; m < 4; m++) {
        if (c->p.sap_block[m] < 2 || (c->p.sap_block[m] & 1) || c->g.L[m] % c->p.sap_block[m] ||
            c->p.sap_block[0] * c->p.sap_block[1] * c->p.sap_block[2] * c->p.sap_block[3] > 256) {
            c->err = "sap_block must be even, divide the lattice extent and hold <= 256 sites";
            return OVL_EINVAL;
        }
    }
    if (!c->sap_tuned) {
        ST(c->autotune_sap());
        c->sap_tuned = true;
    }
    ST(c->import_vec(b, c->io_a));
    int it = 0;
    ST(wilson_solve_eo(c, c->io_a, c->io_b, m0, tol, &it));
    if (iters) *iters = it;
    return c->export_vec(c->io_b, x);
}

extern "C" ovl_status wilson_sap_apply(ovl_ctx *ctx, double *out, const double *in, double m0) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    if (!isfinite(m0)) {
        c->err = "m0 must be finite";
        return OVL_EINVAL;
    }
    for (int m = 0; m < 4; m++) {
        if (c->p.sap_block[m] < 2 || (c->p.sap_block[m] & 1) || c->g.L[m] % c->p.sap_block[m] ||
            c->p.sap_block[0] * c->p.sap_block[1] * c->p.sap_block[2] * c->p.sap_block[3] > 256) {
            c->err = "sap_block must be even, divide the lattice extent and hold <= 256 sites";
            return OVL_EINVAL;
        }
    }
    if (c->p.sap_cycles < 1 || c->p.sap_mr_iters < 1) {
        c->err = "sap_cycles and sap_mr_iters must be >= 1";
        return OVL_EINVAL;
    }
    if (!c->sap_tuned) {
        ST(c->autotune_sap());
        c->sap_tuned = true;
    }
    ST(c->import_vec(in, c->io_a));
    ST(sap_apply_eo(c, c->io_a, c->io_b, m0));
    return c->export_vec(c->io_b, out);
}

// ------------------------------------------------------------------ operators in a chosen arithmetic
static bool arith_ok(int a) {
    return a == OVL_ARITH_FP64 || a == OVL_ARITH_FF || a == OVL_ARITH_FP32 || a == OVL_ARITH_FP16 ||
           a == OVL_ARITH_BF16;
}

extern "C" ovl_status wilson_apply_arith(ovl_ctx *ctx, double *out, const double *in, double m0, int arith) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    if (!isfinite(m0) || !arith_ok(arith)) {
        c->err = "wilson_apply_arith: need finite m0 and an ovl_arith value";
        return OVL_EINVAL;
    }
    ST(c->import_vec(in, c->io_a));
    const long w = (long)c->g.V * 12;
    if (arith == OVL_ARITH_FP64) {
        CK(wilson_f64(c->g, c->U64, c->io_a, c->io_b, m0, 0, 1.0, nullptr, 0.0, c->stream));
    } else if (arith == OVL_ARITH_FF) {
        ST(c->ensure_msff());
        CK(dev_d2ff(c->io_a, c->msff.t, w, c->stream));
        CK(wilson_ff(c->g, c->Uff, c->msff.t, c->msff.y, m0, 0, 1.0, nullptr, 0.0, c->stream));
        CK(dev_ff2d(c->msff.y, c->io_b, w, c->stream));
    } else if (arith == OVL_ARITH_FP16 || arith == OVL_ARITH_BF16) {
        // 16-bit links and spinors, FP32 arithmetic: FP64 -> FP32 -> 16 bits, stencil, and back
        const bool bf = arith == OVL_ARITH_BF16;
        ST(ensure_f32_buffers(c));
        ST(c->ensure_16(bf));
        CK(spinor_d2f(c->g, c->io_a, (float4 *)c->f_a, c->stream));
        CK(spinor_f2h(c->g, (const float4 *)c->f_a, c->h16a, c->h16na, bf, c->stream));
        CK(wilson_16(c->g, c->U16[bf ? 1 : 0], c->h16a, c->h16na, c->h16b, c->h16nb, (float)m0, bf, c->stream));
        CK(spinor_h2f(c->g, c->h16b, c->h16nb, (float4 *)c->f_b, bf, c->stream));
        CK(spinor_f2d(c->g, (const float4 *)c->f_b, c->io_b, c->stream));
    } else {
        ST(ensure_f32_buffers(c));
        CK(spinor_d2f(c->g, c->io_a, (float4 *)c->f_a, c->stream));
        CK(wilson_f32(c->g, c->U32, (const float4 *)c->f_a, (float4 *)c->f_b, (float)m0, 0, 1.f, nullptr, 0.f,
                      c->stream));
        CK(spinor_f2d(c->g, (const float4 *)c->f_b, c->io_b, c->stream));
    }
    return c->export_vec(c->io_b, out);
}

extern "C" ovl_status wilson_apply_n_arith(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double m0,
                                           int arith) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    if (arith == OVL_ARITH_FP64) return wilson_apply_n(ctx, out, in, n_rhs, m0);
    if (n_rhs < 1 || !isfinite(m0) || arith != OVL_ARITH_FP32) {
        c->err = "wilson_apply_n_arith: need n_rhs >= 1, finite m0 and arith OVL_ARITH_FP64 or OVL_ARITH_FP32";
        return OVL_EINVAL;
    }
    const int blk = std::min(kMaxBatch, n_rhs);
    if (!c->xbat || c->xbat_cap < blk) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2 * blk));
        c->xbat = (double2 *)buf;
        c->bbat = c->xbat + (size_t)blk * c->g.V * 12;
        c->xbat_cap = blk;
    }
    if (!c->fbat || c->fbat_cap < blk) {
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(float) * 2 * blk));
        c->fbat = (float *)buf;
        c->fbat_cap = blk;
    }
    const long w = (long)c->g.V * 12, wf = (long)c->g.V * 6;
    float4 *fa = (float4 *)c->fbat, *fb = fa + (size_t)blk * wf;
    for (int r0 = 0; r0 < n_rhs; r0 += blk) {
        const int nb = std::min(blk, n_rhs - r0);
        for (int y = 0; y < nb; y++) ST(c->import_vec(in + (size_t)(r0 + y) * c->n64, c->bbat + y * w));
        CK(spinor_d2f_n(c, c->bbat, fa, nb));
        CK(wilson_batch_f32(c->g, c->U32, fa, fb, wf, nb, (float)m0, 0, 1.f, nullptr, 0.f, c->stream));
        CK(spinor_f2d_n(c, fb, c->xbat, nb));
        for (int y = 0; y < nb; y++) ST(c->export_vec(c->xbat + y * w, out + (size_t)(r0 + y) * c->n64));
    }
    return OVL_OK;
}

extern "C" ovl_status sign_apply_arith(ovl_ctx *ctx, double *out, const double *in, double tol, int arith) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    ST(check_tol(c, tol));
    if (!arith_ok(arith)) {
        c->err = "sign_apply_arith: arith must be an ovl_arith value";
        return OVL_EINVAL;
    }
    ST(c->import_vec(in, c->io_a));
    ovl_status st;
    if (arith == OVL_ARITH_FP64) {
        st = c->sign64(c->io_a, c->io_b, tol, 0);
    } else if (arith == OVL_ARITH_FF) {
        st = c->sign_ff(c->io_a, c->io_b, tol, 0);
    } else {
        ST(ensure_f32_buffers(c));
        CK(spinor_d2f(c->g, c->io_a, (float4 *)c->f_a, c->stream));
        st = c->sign32((const float4 *)c->f_a, (float4 *)c->f_b, tol, 0,
                       arith == OVL_ARITH_FP16 ? 1 : arith == OVL_ARITH_BF16 ? 2 : 0);
        if (st == OVL_OK || st == OVL_ENOCONV) CK(spinor_f2d(c->g, (const float4 *)c->f_b, c->io_b, c->stream));
    }
    if (st != OVL_OK && st != OVL_ENOCONV) return st;
    ST(c->export_vec(c->io_b, out));
    return st;
}

// Seeded pseudo-random fill of n floats in [-1, 1) (a counter hash per element), so that
// the stencil timings run on data of the magnitude of a real field and not on zeros.
__global__ void k_fill_random(float *x, long n, unsigned seed) {
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)k * 2654435761u ^ seed;
        h ^= h >> 16;
        h *= 0x7feb352du;
        h ^= h >> 15;
        h *= 0x846ca68bu;
        h ^= h >> 16;
        x[k] = (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
    }
}
cudaError_t ovl::fill_random_f32(float *x, long n, unsigned seed, cudaStream_t st) {
    k_fill_random<<<std::min<long>(4096, (n + kBlock - 1) / kBlock), kBlock, 0, st>>>(x, n, seed);
    count_launches(1);
    return cudaGetLastError();
}
static cudaError_t fill_random(void *buf, size_t bytes, cudaStream_t st) {
    return fill_random_f32((float *)buf, (long)(bytes / sizeof(float)), 0x9e3779b9u, st);
}

extern "C" ovl_status ovl_dslash_time(ovl_ctx *ctx, int precision, int reps, double *ms) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !ms || reps < 1 || precision < 0 || precision > 4) return OVL_EINVAL;
    if (precision == 2) ST(c->ensure_ff_links());
    if (precision >= 3) {
        ST(ensure_f32_buffers(c));
        ST(c->ensure_16(precision == 4));
    }
    void *buf;
    ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2));
    // random input spinor (floats reinterpreted: FP64 words become finite values of
    // moderate exponent, FP32 and float-float words values in [-1, 1))
    if (precision == 0) {
        CK(fill_random(buf, (size_t)c->n64 * sizeof(double), c->stream));
        CK(spinor_f2d(c->g, (const float4 *)buf, (double2 *)buf + (size_t)c->g.V * 12, c->stream));
        CK(cudaMemcpyAsync(buf, (double2 *)buf + (size_t)c->g.V * 12, (size_t)c->n64 * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(fill_random(buf, (size_t)c->n64 * sizeof(double) * 2, c->stream));
    }
    if (precision >= 3)   // random FP32 spinor rounded to the 16-bit format
        CK(spinor_f2h(c->g, (const float4 *)buf, c->h16a, c->h16na, precision == 4, c->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    ovl_status st = OVL_OK;
    for (int k = 0; k < 3 + reps && st == OVL_OK; k++) {
        if (k == 3 && cudaEventRecord(e0, c->stream) != cudaSuccess) st = OVL_ECUDA;
        cudaError_t e;
        if (precision == 0)
            e = wilson_f64(c->g, c->U64, (const double2 *)buf, (double2 *)buf + (size_t)c->g.V * 12, c->m0_ker, 0, 1.0,
                           nullptr, 0.0, c->stream);
        else if (precision == 2)
            e = wilson_ff(c->g, c->Uff, (const ffw *)buf, (ffw *)buf + (size_t)c->g.V * 12, c->m0_ker, 0, 1.0, nullptr,
                          0.0, c->stream);
        else if (precision >= 3)
            e = wilson_16(c->g, c->U16[precision - 3], c->h16a, c->h16na, c->h16b, c->h16nb, (float)c->m0_ker,
                          precision == 4, c->stream);
        else
            e = wilson_f32(c->g, c->U32, (const float4 *)buf, (float4 *)buf + (size_t)c->g.V * 6, (float)c->m0_ker, 0,
                           1.f, nullptr, 0.f, c->stream);
        if (e != cudaSuccess) st = OVL_ECUDA;
    }
    float t = 0.f;
    if (st == OVL_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = OVL_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), buf));
    if (st != OVL_OK) {
        cudaGetLastError();
        c->err = "ovl_dslash_time: CUDA error";
        return st;
    }
    *ms = t / reps;
    return OVL_OK;
}

extern "C" ovl_status wilson_apply_n(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double m0) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    if (n_rhs < 1 || !isfinite(m0)) {
        c->err = "need n_rhs >= 1 and finite m0";
        return OVL_EINVAL;
    }
    ST(c->ensure_batch());
    if (!c->xbat) {   // staging for one block of right-hand sides (kept; reused by later calls)
        const int cap = std::min(kMaxBatch, n_rhs);
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2 * cap));
        c->xbat = (double2 *)buf;
        c->bbat = c->xbat + (size_t)cap * c->g.V * 12;
        c->xbat_cap = cap;
    }
    const int blk = c->xbat_cap;
    const long w = (long)c->g.V * 12;
    for (int r0 = 0; r0 < n_rhs; r0 += blk) {
        const int nb = std::min(blk, n_rhs - r0);
        for (int y = 0; y < nb; y++) ST(c->import_vec(in + (size_t)(r0 + y) * c->n64, c->bbat + y * w));
        CK(wilson_batch_f64(c->g, c->U64, c->bbat, c->xbat, w, nb, m0, 0, 1.0, nullptr, 0.0, c->stream));
        for (int y = 0; y < nb; y++) ST(c->export_vec(c->xbat + y * w, out + (size_t)(r0 + y) * c->n64));
    }
    return OVL_OK;
}

extern "C" ovl_status ovl_apply_n(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double tol) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    ST(check_ctx_ptrs(c, out, in));
    ST(check_tol(c, tol));
    if (n_rhs < 1) {
        c->err = "n_rhs must be >= 1";
        return OVL_EINVAL;
    }
    ST(c->ensure_batch());
    if (!c->xbat) {   // staging for one block of right-hand sides (kept; reused by later calls)
        const int cap = std::min(kMaxBatch, n_rhs);
        void *buf;
        ST(c->alloc(&buf, (size_t)c->n64 * sizeof(double) * 2 * cap));
        c->xbat = (double2 *)buf;
        c->bbat = c->xbat + (size_t)cap * c->g.V * 12;
        c->xbat_cap = cap;
    }
    const int blk = c->xbat_cap;
    const long w = (long)c->g.V * 12;
    double t[kMaxBatch];
    for (int y = 0; y < kMaxBatch; y++) t[y] = tol;
    for (int r0 = 0; r0 < n_rhs; r0 += blk) {
        const int nb = std::min(blk, n_rhs - r0);
        for (int y = 0; y < nb; y++) ST(c->import_vec(in + (size_t)(r0 + y) * c->n64, c->bbat + y * w));
        ST(c->sign64_batch(c->bbat, c->xbat, nb, t, 1));
        for (int y = 0; y < nb; y++) ST(c->export_vec(c->xbat + y * w, out + (size_t)(r0 + y) * c->n64));
    }
    return OVL_OK;
}

extern "C" ovl_status ovl_dslash_time_n(ovl_ctx *ctx, int precision, int nrhs, int reps, double *ms) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || !ms || reps < 1 || nrhs < 1 || nrhs > kMaxBatch || (precision != 0 && precision != 1)) return OVL_EINVAL;
    void *buf;
    const size_t bytes = (size_t)c->n64 * (precision == 0 ? 8 : 4) * nrhs * 2;
    ST(c->alloc(&buf, bytes));
    if (precision == 0) {   // FP64 random values: FP32 random words converted, one vector at a time
        const long w = (long)c->g.V * 12;
        CK(fill_random(buf, (size_t)c->n64 * sizeof(double), c->stream));
        for (int y = 1; y < 2 * nrhs; y++)
            CK(spinor_f2d(c->g, (const float4 *)buf, (double2 *)buf + y * w, c->stream));
        CK(cudaMemcpyAsync(buf, (double2 *)buf + w, (size_t)w * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(fill_random(buf, bytes, c->stream));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    ovl_status st = OVL_OK;
    for (int k = 0; k < 3 + reps && st == OVL_OK; k++) {
        if (k == 3 && cudaEventRecord(e0, c->stream) != cudaSuccess) st = OVL_ECUDA;
        cudaError_t e;
        if (precision == 0) {
            const long w = (long)c->g.V * 12;
            e = wilson_batch_f64(c->g, c->U64, (const double2 *)buf, (double2 *)buf + w * nrhs, w, nrhs, c->m0_ker, 0,
                                 1.0, nullptr, 0.0, c->stream);
        } else {
            const long w = (long)c->g.V * 6;
            e = wilson_batch_f32(c->g, c->U32, (const float4 *)buf, (float4 *)buf + w * nrhs, w, nrhs,
                                 (float)c->m0_ker, 0, 1.f, nullptr, 0.f, c->stream);
        }
        if (e != cudaSuccess) st = OVL_ECUDA;
    }
    float t = 0.f;
    if (st == OVL_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = OVL_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), buf));
    if (st != OVL_OK) {
        cudaGetLastError();
        c->err = "ovl_dslash_time_n: CUDA error";
        return st;
    }
    *ms = t / reps;
    return OVL_OK;
}

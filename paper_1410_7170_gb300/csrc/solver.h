// Library context and the host-side solver interfaces (internal).
#pragma once
#include <chrono>
#include <complex>
#include <string>
#include <vector>

#include "../../include/ovl.h"
#include "internal.h"
#include "mg.h"

namespace ovl {

// Status propagation inside Ctx members and helpers (a Ctx *c must be in scope for CK):
// CK turns a CUDA error into OVL_ECUDA with the failing call recorded in c->err (and the
// sticky last-error cleared); ST returns any non-OK ovl_status.
#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            cudaGetLastError();                                                    \
            c->err = std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #expr; \
            return OVL_ECUDA;                                                      \
        }                                                                          \
    } while (0)
#define ST(expr)                     \
    do {                             \
        ovl_status s_ = (expr);      \
        if (s_ != OVL_OK) return s_; \
    } while (0)


struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    int chunk = 0;
    bool prof = false;
    int nrhs = 0;
};

constexpr int kMaxChunk = 64;
constexpr int kScal = 8192;   // doubles of scalar staging (device d_scal, pinned h_scal)

// Event timings of the multishift kernels (instrumentation).
struct ProfAcc {
    double q_ms = 0, r_ms = 0, s_ms = 0;           // event time of the timed launches
    long q_t = 0, r_t = 0, s_t = 0;                // timed launches
    double q_tb = 0, r_tb = 0, s_tb = 0;           // their algorithmic bytes
    long n = 0;                                    // iterations (launches of each kernel)
    double q_bytes = 0, r_bytes = 0, s_bytes = 0;  // algorithmic bytes of all launches
    bool valid = true;
};

// A Krylov basis workspace: V (m+1 vectors), Z (m vectors, flexible only), w, r.
template <typename T>
struct Krylov {
    T *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
    int m = 0;
    bool flexible = false;
};

struct Ctx {
    // geometry and operator parameters
    Geom g{};
    long n64 = 0;                 // reals per spinor (24 V)
    double rho_in = 1, mu = 0, rho = 1, m0_ker = -1, m0_prec = 0, sigma_min = 0;
    ovl_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // memory
    std::vector<void *> allocs;
    size_t bytes_held = 0;
    void *h_pinned = nullptr;
    double *h_scal = nullptr;     // pinned scalars (kScal doubles; coefficient staging in the upper half)
    int *h_flag = nullptr;
    int *h_ms_small = nullptr;
    MsState *h_ms = nullptr;
    RedScratch rs{};
    int *d_flag = nullptr;
    double *d_scal = nullptr;
    double *d_md_part = nullptr;  // multi-dot partials
    double *d_coef = nullptr;     // multi-axpy coefficients
    // gauge field (12-real links)
    double2 *U64 = nullptr;
    float4 *U32 = nullptr;
    ffw *Uff = nullptr;           // float-float copy of U64 (made on first use)
    void *U16[2] = {nullptr, nullptr};    // 16-bit links: FP16 [0], BF16 [1] (made on first use)
    uint4 *h16a = nullptr, *h16b = nullptr;   // two 16-bit spinors (48 B per site)
    float *h16na = nullptr, *h16nb = nullptr; // their per-site FP16 scales
    // boundary staging
    double *io_lex = nullptr;
    double2 *io_a = nullptr, *io_b = nullptr;
    // Zolotarev
    int npole = 0;
    double lam_min = 0, lam_max = 0, zd0 = 0, zdelta = 0;
    // Zolotarev coefficients of every degree n = 1..npole (index n - 1) on [lam_min, lam_max]
    std::vector<double> zs_d0, zs_delta;
    std::vector<std::vector<double>> zs_a, zs_c;
    bool lam_estimated = false;
    std::vector<double> za, zc;
    // multishift
    MsState *ms64_state = nullptr, *ms32_state = nullptr;
    MsVectors<double2> ms64{};
    MsVectors<float4> ms32{};
    MsVectorsH msh{};
    MsState *msh_state = nullptr;
    MsVectors<ffw> msff{};             // float-float multishift vectors
    MsState *msff_state = nullptr;
    GraphSlot graphs[8];
    // batched multishift (several right-hand sides in lock-step)
    MsBatch<double2> msb64{};
    MsBatch<float4> msb32{};
    int msb64_cap = 0, msb32_cap = 0;
    MsState *msb_state = nullptr;      // kMaxBatch states
    MsState *h_msb = nullptr;          // pinned host copies
    int *h_msb_small = nullptr;        // pinned: 4 ints per state
    RedScratch rsb{};                  // per-row partials for batched reductions
    unsigned *bcounters = nullptr;     // per-row arrival counters
    void *h_pinned_b = nullptr;
    // instrumentation
    bool prof = false;
    ProfAcc pacc[3];   // per arithmetic slot (0 FP64, 1 FP32 / 16-bit stored, 2 float-float)
    long launch_mark = 0;
    cudaEvent_t ev[3][4] = {};   // profiling: events around the kernels of one sampled iteration
    bool ev_ready[3] = {false, false, false};
    int *d_hist = nullptr;
    int hist_cap = 0;
    int *h_hist = nullptr;
    // Krylov workspaces
    Krylov<double> kry_outer, kry_wil64;
    Krylov<float> kry_inner, kry_wil32;
    Krylov<double> kbo_outer, kbo_wil64;   // batched: N vectors per basis entry
    Krylov<float> kbo_inner, kbo_wil32;
    int kb_n[4] = {0, 0, 0, 0};
    float *fbat = nullptr;             // FP32 staging of a batch (2 x nb vectors)
    int fbat_cap = 0;
    double2 *xbat = nullptr, *bbat = nullptr;   // FP64 batch of solutions / right-hand sides
    int xbat_cap = 0;
    float *f_a = nullptr, *f_b = nullptr;   // FP32 conversion buffers
    void *sap_r32 = nullptr, *sap_r64 = nullptr;   // SAP residual scratch
    double2 *d_x = nullptr, *d_b = nullptr; // FP64 solve vectors
    // statistics of the running call
    long stat_ms64 = 0, stat_ms32 = 0, stat_msff = 0, stat_prec = 0;
    int stat_inner = 0;
    float tune_ms[4] = {0, 0, 0, 0};   // stencil ms: fp64 1/4 tps, fp32 1/4 tps
    float tune_mrhs_ms[6] = {0, 0, 0, 0, 0, 0};   // FP32 multi-RHS stencil ms per RHS of kernels 1, 2, 3
                                                    // at 4 right-hand sides, then at 12
    int sap_tps = 1;                   // threads per site of the FP32 Schwarz block kernel
    double t_sign64 = 0, t_sign_low = 0, t_prec = 0;   // phase wall times of the current solve (s)
    bool sap_tuned = false;
    float sap_ms[3] = {0, 0, 0};       // one FP32 Schwarz cycle, ms: 1, 2, 4 threads per site
    // low-mode deflation of the sign function (params.n_deflate > 0)
    int ndefl = 0;
    double2 *defl64 = nullptr, *defl64g5 = nullptr;   // eigenvectors xi_i of Q and gamma5 xi_i (FP64)
    float4 *defl32 = nullptr, *defl32g5 = nullptr;    // the same in FP32
    double2 *defl_tmp64 = nullptr;                    // projected right-hand side
    float4 *defl_tmp32 = nullptr;
    std::vector<double> defl_lambda;                  // eigenvalues of the deflated pairs (signed)
    double defl_next = 0, defl_setup_s = 0, defl_resid = 0;   // |lambda_{k+1}|, seconds, max ||Q xi - lambda xi||
    long defl_matvecs = 0;                            // Q^2 applications of the eigensolver
    // restarted Krylov sign function (params.sign_method == OVL_SIGN_KRYLOV)
    double2 *ks_W = nullptr, *ks_Y = nullptr;         // basis (krylov_m + 1 vectors), kept Ritz vectors
    double2 *ks_f = nullptr, *ks_tmp = nullptr;       // accumulated f(Q^2) Q b, stencil scratch
    double *ks_S = nullptr;                           // Ritz coefficients (device)
    long ks_cycles = 0, ks_matvecs = 0;               // totals since creation
    // two-level multigrid for the Wilson solves (params.wilson_mg)
    MgData mg;
    // On-the-fly choice of the Wilson preconditioner mass of the inner FGMRES (params.m0_adapt):
    // candidate masses around m0^def, each scored by the residual reduction of the inner
    // FGMRES iteration its preconditioner application served, per second of that iteration.
    struct M0Adapt {
        std::vector<double> cand, gain, cost;
        std::vector<long> n;
        int pending = -1;                    // candidate of the last application, not yet scored
        double rel_pending = 0;              // relative residual before that application
        std::chrono::steady_clock::time_point t_pending{};
        uint64_t rng = 0x2545F4914F6CDD1Dull;
        long uses = 0;
    } m0a;
    double fgmres_rel = -1;   // relative residual estimate of the FGMRES calling the preconditioner
    // batches of several right-hand sides sized by params.rhs_block alone, not by the free
    // device memory (set by the serving loop, which reserves that memory at admission, so
    // that a request's batching does not depend on what else is running)
    bool fixed_batch = false;
    // wall-clock limit of the running ovl_solve (params.max_seconds; 0 = none)
    std::chrono::steady_clock::time_point deadline{};
    bool has_deadline = false;
    // true (with err set) once the running solve is past its wall-clock limit
    bool past_deadline() {
        if (!has_deadline || std::chrono::steady_clock::now() < deadline) return false;
        err = "ovl_solve: wall-clock limit params.max_seconds reached";
        return true;
    }

    ~Ctx();
    ovl_status alloc(void **p, size_t bytes);
    ovl_status sync();
    ovl_status fetch(const double *d, int n, double *h);
    ovl_status norm2_d(const double *x, double *out);
    ovl_status norm2_f(const float *x, double *out);
    ovl_status import_vec(const double *src, double2 *dst);
    ovl_status export_vec(const double2 *src, double *dst);
    int pick_poles(double tol) const;
    void fill_poles(MsState &s, int n, double tol) const;
    ovl_status ms_setup(MsState *d_state, double tol, int *n_out);
    // which: instrumentation class (0 FP64, 1 FP32/FP16); slot: CUDA-graph slot;
    // shift_bytes: algorithmic bytes per site of one shift update (read + write of p_l)
    template <typename Iter>
    ovl_status ms_run(MsState *d_state, int which, int slot, double shift_bytes, bool fused, Iter iter_fn,
                      int *iters_out);
    ovl_status sign64(const double2 *b, double2 *out, double tol, int mode);
    // store: -1 = from params.precision, 0 = FP32, 1 = FP16-stored, 2 = BF16-stored directions
    ovl_status sign32(const float4 *b, float4 *out, double tol, int mode, int store = -1);
    // the FP64-accuracy sign in float-float arithmetic on FP64 even-odd vectors b, out
    ovl_status sign_ff(const double2 *b, double2 *out, double tol, int mode);
    ovl_status ensure_ff_links();
    ovl_status ensure_16(bool bf16);   // 16-bit links of the requested type and two 16-bit spinors
    ovl_status ensure_msff();
    // FP64-accuracy sign of the outer solver: float-float in the mixed precisions when
    // params.ff_outer is set, native FP64 otherwise
    ovl_status sign_outer(const double2 *b, double2 *out, double tol, int mode);
    ovl_status sign64_krylov(const double2 *b, double2 *out, double tol, int mode);
    ovl_status ensure_ksign();
    ovl_status ensure_ms64();
    ovl_status ensure_ms32();
    ovl_status ensure_msh();
    // several right-hand sides: b, out hold nrhs internal vectors back to back
    ovl_status ensure_batch();
    ovl_status sign64_batch(const double2 *b, double2 *out, int nrhs, const double *tol, int mode);
    ovl_status sign_outer_batch(const double2 *b, double2 *out, int nrhs, const double *tol, int mode);
    ovl_status sign32_batch(const float4 *b, float4 *out, int nrhs, const double *tol, int mode);
    template <typename ST, typename Init, typename Iter>
    ovl_status msb_run(int nrhs, const double *tol, int n, int slot, Init init_fn, Iter iter_fn, long *iters_out);
    ovl_status lanczos_bounds(double *lmin, double *lmax, double m0 = NAN);   // |eigenvalues| of Q(m0), default m0_ker
    ovl_status sigma_min_estimate(double *smin);
    ovl_status set_zolotarev();
    ovl_status autotune();
    ovl_status autotune_mrhs();
    ovl_status autotune_sap();
    ovl_status deflation_setup();
    ovl_status defl_project64(const double2 *b, double2 *bp, std::vector<double> &coef);
    ovl_status defl_add64(const std::vector<double> &coef, double2 *out, int mode);
    ovl_status defl_project32(const float4 *b, float4 *bp, std::vector<double> &coef);
    ovl_status defl_add32(const std::vector<double> &coef, float4 *out, int mode);
};

// Wall time of a solver phase, added to *acc when the scope ends. With profiling on, the
// context's stream is synchronised first, so that the phase's last kernels are counted.
struct PhaseClock {
    Ctx *c;
    double *acc;
    std::chrono::steady_clock::time_point t0;
    PhaseClock(Ctx *c_, double *a) : c(c_), acc(a), t0(std::chrono::steady_clock::now()) {}
    ~PhaseClock() {
        if (c->prof) cudaStreamSynchronize(c->stream);
        *acc += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Complex coefficients (interleaved) to c->d_coef through the pinned staging area; the
// caller makes sure the previous upload has completed (a fetch in between synchronises).
ovl_status upload_coef(Ctx *c, const std::vector<std::complex<double>> &v);

ovl_status solve_all(Ctx *c, double *x, const double *b, int n_rhs, double tol, ovl_stats *stats);
// FP32 conversion buffers f_a, f_b (one spinor each), allocated on first use
ovl_status ensure_f32_buffers(Ctx *c);
// FP64 <-> FP32 even-odd conversion of nb spinors back to back
cudaError_t spinor_d2f_n(Ctx *c, const double2 *a, float4 *b, int nb);
cudaError_t spinor_f2d_n(Ctx *c, const float4 *a, double2 *b, int nb);
// Lock-step batched solve of nrhs <= kMaxBatch systems on internal FP64 vectors.
ovl_status solve_batch(Ctx *c, double2 *x, const double2 *b, int nrhs, double tol, int *outer_iters,
                       double *worst_res, bool *all_conv);
// Inexact Wilson solve on FP64 even-odd spinors (FP32 inside unless precision == FP64).
ovl_status wilson_solve_eo(Ctx *c, const double2 *b, double2 *x, double m0, double tol, int *iters);
// One Schwarz preconditioner application x = M_SAP b on FP64 even-odd spinors.
ovl_status sap_apply_eo(Ctx *c, const double2 *b, double2 *x, double m0);
// Two-level multigrid for D_W(m0) (mg_ctl.cu): setup from n_start start vectors (boundary
// layout; NULL = seeded pseudo-random ones), and one preconditioner application on FP32
// even-odd spinors (the setup is made, or remade for a new m0, first).
ovl_status mg_setup(Ctx *c, double m0, const double *start, int n_start);
ovl_status mg_apply_f32(Ctx *c, const float4 *r, float4 *x, double m0);

}  // namespace ovl

/* ovl.h — C ABI of the GB300 overlap-operator library (libovl.so).
 *
 * The library applies and inverts Neuberger's overlap operator
 *
 *     D_N = rho I + Gamma5 sign(Gamma5 D_W(m0_ker))          (Sec. 2, Eq. overlap_def)
 *
 * with the Wilson-Dirac kernel D_W of Eq. (Wilson-Dirac) (lattice spacing a = 1),
 * kernel mass m0_ker = -rho_in and rho = (-mu/2 + m0_ker)/(mu/2 + m0_ker) (Sec. 5).
 * sign(Q), Q = Gamma5 D_W, is evaluated with Zolotarev's optimal rational
 * approximation on [lambda_min, lambda_max] of |Q| and a multishift conjugate
 * gradient for the shifted systems (Q^2 + sigma_l) x_l = b, or (params.sign_method)
 * by the restarted Krylov method with thick restarts of Sec. 5.2. D_N psi = eta
 * (Eq. linsys) is solved by restarted GMRES(m) or right-preconditioned
 * FGMRES(m) in FP64 (Sec. 5.1), optionally with relaxation of the sign
 * accuracy (Sec. 5.2) and a Wilson-Dirac preconditioner D_W(m0_prec)^{-1}
 * (Sec. 3, Eq. default_m), applied inexactly (Sec. 5.1) or inside a nested
 * FP32 inner FGMRES on D_N (Sec. 5.3).
 *
 * Field layout at the boundary (every vector argument):
 *   lattice dims[4] = {L0, L1, L2, L3}, x0 = time; all L_mu even and >= 2;
 *   lexicographic site index s = ((x0*L1 + x1)*L2 + x2)*L3 + x3;
 *   spinor: V*12 complex doubles, interleaved (re, im), ordered [s][spin][colour]
 *           (gamma matrices in the chiral basis gamma_0 = [[0,I],[I,0]],
 *            gamma_k = [[0,-i sigma_k],[i sigma_k,0]], gamma_5 = diag(-1,-1,1,1));
 *   several right-hand sides are n_rhs such vectors back to back;
 *   gauge: V*4*9 complex doubles ordered [s][mu][row][col], U_mu(x) links x -> x+mu,
 *          each an SU(3) matrix.
 * Pointers may be device memory or host memory (pageable or pinned); the
 * library detects which and copies host data in and out itself. The caller owns
 * every buffer it passes; the library keeps no pointer to them after a call
 * returns. A context owns all its device memory (gauge copies, workspace).
 *
 * Errors: every call returns an ovl_status; nothing aborts, traps or throws across
 * the ABI. On error the output buffers are unspecified and ovl_last_error() gives
 * a one-line reason. Calls on one context are ordered on the context's CUDA stream
 * and return after the stream has finished the call's work; one context must not be
 * used from two threads at once (different contexts may).
 */
#ifndef OVL_H
#define OVL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ovl_ctx ovl_ctx;

typedef enum {
    OVL_OK = 0,
    OVL_EINVAL = 1,       /* bad argument (size, pointer, non-SU(3) link, NaN input) */
    OVL_ENOMEM = 2,       /* device memory / HBM budget exhausted */
    OVL_ENOCONV = 3,      /* iteration cap reached before the tolerance */
    OVL_EBREAKDOWN = 4,   /* Krylov breakdown (zero or non-finite scalar) */
    OVL_ETIMEOUT = 5,     /* ovl_solve passed its wall-clock limit (params.max_seconds) */
    OVL_ECUDA = 6         /* CUDA runtime error */
} ovl_status;

typedef enum {
    OVL_FP64 = 0,         /* everything in FP64 */
    OVL_MIXED_FP32 = 1,   /* inner (preconditioner) work in FP32, outer D_N in FP64 */
    OVL_MIXED_HALF = 2,   /* as MIXED_FP32, inner multishift vectors stored in FP16 */
    OVL_MIXED_BF16 = 3    /* as MIXED_FP32, inner multishift vectors stored in BF16 */
} ovl_precision;

/* Arithmetic of one operator application through the *_arith entry points (the solver's
 * own choice follows ovl_params.precision and ff_outer). */
typedef enum {
    OVL_ARITH_FP64 = 0,   /* FP64 storage and arithmetic */
    OVL_ARITH_FF = 1,     /* float-float: each real is an unevaluated sum of two FP32 numbers (about
                             48 significant bits), computed on the FP32 pipes; same bytes as FP64 */
    OVL_ARITH_FP32 = 2,   /* FP32 storage and arithmetic (links stored as 12 reals) */
    OVL_ARITH_FP16 = 3,   /* FP32 arithmetic on 16-bit data. Stencil: links (12 reals) and spinors in
                             FP16, spinors with a per-site FP32 scale. Sign: the multishift's shifted
                             directions stored in FP16 with a per-site scale */
    OVL_ARITH_BF16 = 4    /* as OVL_ARITH_FP16 with BF16 storage (no scale) */
} ovl_arith;

typedef enum {
    OVL_PREC_NONE = 0,      /* GMRES(m), no preconditioner (Sec. 5.1 baseline) */
    OVL_PREC_WILSON = 1,    /* FGMRES(m) right-preconditioned by an inexact D_W(m0_prec)^{-1} (Sec. 5.1) */
    OVL_PREC_RECURSIVE = 2  /* FGMRES(m) preconditioned by an inner FP32 FGMRES on D_N, itself
                               preconditioned by the inexact Wilson solve (Sec. 5.3) */
} ovl_precond;

typedef enum {
    OVL_SIGN_ZOLOTAREV = 0, /* Zolotarev rational approximation evaluated by multishift CG */
    OVL_SIGN_KRYLOV = 1     /* restarted Krylov method with thick restarts (Sec. 5.2, FP64 only) */
} ovl_sign_method;

/* Solver and approximation parameters. Defaults (ovl_params_default) are the
 * paper's Table 2 / Table 3 values where the paper gives one. */
typedef struct {
    double tol_outer;       /* relative residual target ||b - D_N x|| / ||b|| (Table 2: 1e-8) */
    int restart;            /* (F)GMRES restart length m (Table 2: 100) */
    int relax;              /* 1: sign accuracy relaxed to tol_outer/||r_k||_rel * relax_factor (Sec. 5.2) */
    double relax_factor;    /* Table 2: 1e-2 */
    int n_poles;            /* Zolotarev poles n, the largest degree used (1..64; default 20) */
    double lambda_min;      /* spectral interval of |Q|; 0 = estimate by Lanczos at ovl_create */
    double lambda_max;
    double sign_tol;        /* accuracy of sign_apply inside ovl_apply/ovl_solve when relax = 0 */
    int precond;            /* ovl_precond */
    double m0_prec;         /* Wilson preconditioner mass; NaN = m0^def of Eq. (default_m) */
    double eps_prec;        /* relative residual of the inexact Wilson solve (Table 2: 1e-1) */
    double eps_inner;       /* inner FGMRES residual reduction (Table 3: 1e-2 with preconditioning) */
    int restart_inner;      /* inner FGMRES restart length (Table 3: 100) */
    int max_inner;          /* cap on inner FGMRES iterations per application */
    int precision;          /* ovl_precision */
    int antiperiodic;       /* 1: antiperiodic time boundary for the fermions, 0: periodic */
    int max_iter;           /* cap on outer iterations */
    int max_ms_iter;        /* cap on multishift CG iterations per sign application */
    int sap_block[4];       /* Schwarz block extent (default 4,4,4,4); with a preconditioner each must be even and divide L_mu */
    int sap_cycles;         /* Schwarz cycles per preconditioner application */
    int sap_mr_iters;       /* minimal-residual steps per block solve */
    int prec_restart;       /* restart length of the Wilson FGMRES in the inexact solve */
    int prec_max_iter;      /* cap on Wilson FGMRES iterations per application */
    int rhs_block;          /* right-hand sides solved in lock-step by ovl_solve (1..12; default 4, the
                               fastest measured at 16^4 with 12 right-hand sides; 1 = one after another) */
    int use_graphs;         /* 1: capture multishift iterations in CUDA graphs */
    int check_every;        /* multishift iterations between host convergence checks */
    int stencil_tps;        /* threads per lattice site of the stencils: 0 = autotune, 1 or 4 = forced */
    int sap_tps;            /* threads per block site of the FP32 Schwarz block solves: 0 = autotune, 1, 2 or 4 */
    int adaptive_poles;     /* 1 (default): each sign application uses the smallest Zolotarev degree
                               n <= n_poles whose uniform error delta(k, n) is <= 1/10 of its requested
                               accuracy; 0: always n_poles */
    int n_deflate;          /* k > 0: deflate the k eigenpairs of Q of smallest |lambda| (Sec. 5.2):
                               computed once at ovl_create (FP64 thick-restart Krylov-Schur on Q^2),
                               applied exactly, the sign iteration runs on the projected vector and its
                               interval starts at 0.9 |lambda_{k+1}|. 0 (default): no deflation; <= 48 */
    double deflate_tol;     /* eigenpair accuracy: Ritz residual of Q^2 <= deflate_tol * lambda_max^2
                               (default 1e-13) */
    int sign_method;        /* ovl_sign_method of every FP64 sign application (sign_apply, ovl_apply, the
                               outer D_N of ovl_solve); FP32/FP16/BF16 inner applications always use
                               Zolotarev. Default OVL_SIGN_ZOLOTAREV. OVL_SIGN_KRYLOV computes
                               sign(Q) b = (Q^2)^{-1/2} Q b by restarted Lanczos on Q^2 with
                               quadrature-based restarts (the integral (2/pi) int ds/(Q^2 + s^2)
                               by the trapezoidal rule in ln s) and stops when its error bound
                               (from lambda_min) is <= tol ||b||; right-hand sides run one at a time */
    int krylov_m;           /* basis vectors per cycle of the Krylov sign (4..120; default 40) */
    int krylov_keep;        /* Ritz vectors of the smallest Ritz values of Q^2 kept at a restart
                               (thick restart; 0 = plain restart; <= krylov_m - 2; default 8) */
    int ff_outer;           /* 1 (default): in the mixed precisions (precision != OVL_FP64) the outer
                               solver's sign applications that need more than FP32 accuracy run in
                               float-float arithmetic (OVL_ARITH_FF) instead of native FP64; the
                               outer residuals, Arnoldi vectors and reductions stay FP64. 0: native
                               FP64 for them. Ignored with precision == OVL_FP64 */
    double max_seconds;     /* wall-clock limit of one ovl_solve call (0 = none, the default): checked on
                               the host after every chunk of multishift iterations; past it the call
                               returns OVL_ETIMEOUT (x unspecified) and the context stays usable */
    int wilson_mg;          /* preconditioner of the FP32 Wilson FGMRES (the inexact D_W^{-1} of Sec. 5.1):
                               0 (default) the Schwarz smoother alone; 1 the two-level aggregation
                               multigrid the paper uses (DD-alpha-AMG, two levels, Table 2): aggregates =
                               sap_block blocks split by chirality, mg_nv test vectors from an adaptive
                               setup, coarse GMRES, Schwarz post-smoothing. Needs two or more blocks per
                               direction. FP64 Wilson solves keep the Schwarz preconditioner */
    int mg_nv;              /* test vectors (coarse dofs per aggregate; 1..24, default 12) */
    int mg_setup_iters;     /* smoothing passes v <- v - M_SAP D_W v of the setup (default 4) */
    int mg_coarse_steps;    /* GMRES steps of a coarse solve (1..64, default 16) */
    double mg_coarse_tol;   /* a coarse solve stops early at this relative residual (default 0.1) */
    int m0_adapt;           /* 1: choose the Wilson preconditioner mass of the inner FGMRES (precond =
                               OVL_PREC_RECURSIVE, one right-hand side at a time) on the fly, from one
                               FGMRES iteration to the next (Sec. 5.1): five candidates evenly over
                               [1.5 m0_prec, 0], each scored by the drop of the residual
                               estimate per second of the iteration it served; the scores persist in
                               the context across solves. 0 (default): always m0_prec */
    int mrhs_kernel;        /* FP32 multi-RHS stencil (wilson_apply_n_arith, the FP32 batched paths):
                               0 (default) chosen by the autotuner per lattice shape and block size
                               (up to 6 right-hand sides, 7..12; see ovl_tuning_mrhs), 1 = right-hand
                               sides in pairs looped inside each site's thread, 2 = blocks of 32 sites x
                               one warp per right-hand side, 3 = each site's eight links staged in
                               shared memory once, right-hand sides looped inside the thread */
} ovl_params;

/* Per-solve statistics (all fields written by ovl_solve when stats != NULL). */
typedef struct {
    int outer_iters;        /* outer (F)GMRES iterations, summed over right-hand sides */
    int inner_iters;        /* inner FGMRES iterations (recursive mode) */
    long ms_iters_fp64;     /* multishift CG iterations in FP64 sign applications (with
                               OVL_SIGN_KRYLOV: its products with Q^2) */
    long ms_iters_low;      /* multishift CG iterations in FP32/FP16 sign applications */
    long prec_iters;        /* Wilson FGMRES iterations inside the preconditioner */
    double true_rel_resid;  /* max over RHS of ||b - D_N x|| / ||b||, recomputed in FP64 at exit */
    double seconds;         /* wall time of the call */
    double t_sign_fp64;     /* wall time inside FP64 sign applications (single-RHS path) */
    double t_sign_low;      /* wall time inside FP32/FP16/BF16 sign applications (single-RHS path) */
    double t_prec;          /* wall time inside inexact Wilson solves (single-RHS path); the rest
                               of `seconds` is (F)GMRES orthogonalisation and host work. The phase
                               times are exact (stream synchronised at each phase end) only while
                               ovl_prof_enable is on. t_sign_fp64 includes the float-float sign. */
    long ms_iters_ff;       /* multishift CG iterations of FP64-accuracy sign applications run in
                               float-float arithmetic (params.ff_outer) */
} ovl_stats;

/* Fills *p with the defaults. Returns OVL_EINVAL if p is NULL. */
ovl_status ovl_params_default(ovl_params *p);

/* Creates a context for the lattice dims with kernel mass m0_ker = -rho_in and
 * overlap mass mu (> 0): rho = (rho_in + mu/2)/(rho_in - mu/2) (Sec. 5 with m0_ker = -rho_in).
 * gauge: V*4*9 complex doubles (see layout); copied and compressed to 12 reals per
 * link; links that are not SU(3) to 1e-10 are rejected with OVL_EINVAL.
 * p: NULL = defaults. cuda_stream: a cudaStream_t the context issues all work on
 * (NULL = the context creates its own non-blocking stream).
 * If lambda_min/lambda_max are 0 they are estimated here by Lanczos on Q^2.
 * The Wilson preconditioner mass defaults to m0^def (Eq. default_m). sigma_min, the
 * smallest real part of the eigenvalues of D_W(0), is estimated by the smallest singular
 * value of D_W(0) (Lanczos on (Gamma5 D_W(0))^2).
 * On success *ctx is a new context; on error *ctx is NULL. */
ovl_status ovl_create(ovl_ctx **ctx, const double *gauge, const int dims[4],
                      double rho_in, double mu, const ovl_params *p, void *cuda_stream);

/* out = D_W(m0) in, Eq. (Wilson-Dirac) (one spinor, any m0). */
ovl_status wilson_apply(ovl_ctx *ctx, double *out, const double *in, double m0);

/* x ~= D_W(m0)^{-1} b to relative residual tol: FGMRES(prec_restart) on D_W(m0), right-
 * preconditioned by params.sap_cycles red-black Schwarz cycles over params.sap_block blocks
 * (block solves by params.sap_mr_iters minimal-residual steps), at most params.prec_max_iter
 * iterations; FP32 unless params.precision == OVL_FP64. This is the inexact Wilson solve the
 * overlap solver uses as its preconditioner D_W(m0_prec)^{-1} (Sec. 3, Sec. 5.1). iters
 * (nullable) receives the FGMRES iteration count. Needs even sap_block extents dividing dims. */
ovl_status wilson_solve(ovl_ctx *ctx, double *x, const double *b, double m0, double tol, int *iters);

/* out = M_SAP in, one application of the Schwarz preconditioner that wilson_solve (and the
 * overlap solver's Wilson preconditioner) uses, on D_W(m0): params.sap_cycles red-black
 * multiplicative Schwarz cycles from out = 0 over blocks of params.sap_block sites, coloured
 * by the parity of their block coordinates (colour 0 first); per colour the residual
 * in - D_W out is formed once and every block of that colour adds params.sap_mr_iters
 * minimal-residual steps on its block-local D_W (hops leaving the block dropped). The
 * paper's smoother is a red-black multiplicative Schwarz method (Sec. 5.1) whose block
 * solver it does not specify. FP32 unless params.precision == OVL_FP64. OVL_EINVAL for
 * sap_block extents that are odd, do not divide dims or exceed 256 sites, and for
 * sap_cycles or sap_mr_iters < 1. */
ovl_status wilson_sap_apply(ovl_ctx *ctx, double *out, const double *in, double m0);

/* Stencil variant chosen by the autotuner (threads per site, 1 or 4, for FP64 and FP32)
 * and the measured ms per full-lattice stencil application of each variant
 * (ms[0..3] = FP64 x1, FP64 x4, FP32 x1, FP32 x4; zeros when forced). Nullable outputs. */
ovl_status ovl_tuning(const ovl_ctx *ctx, int *tps64, int *tps32, float *ms);

/* FP32 multi-RHS stencil kernels chosen for this lattice shape (params.mrhs_kernel numbering,
 * 1..3): kernel[0] for blocks of up to 6 right-hand sides, kernel[1] for 7..12; and the
 * autotuner's measured ms per right-hand side of each candidate, ms[0..2] at 4 right-hand sides
 * and ms[3..5] at 12 (kernels 1..3; zeros when params.mrhs_kernel forced the choice). The
 * choice is an implementation detail of the multi-RHS stencil (the paper has no counterpart).
 * Nullable outputs (kernel: 2 ints, ms: 6 floats). */
ovl_status ovl_tuning_mrhs(const ovl_ctx *ctx, int *kernel, float *ms);

/* Deflation state (Sec. 5.2): k deflated pairs, their eigenvalues lambda[k] (signed, by
 * increasing modulus; nullable), |lambda_{k+1}| (the new lower end of the sign interval),
 * the setup time in seconds, max_i ||Q xi_i - lambda_i xi_i|| and the Q^2 applications the
 * eigensolver needed. k = 0 without deflation. */
ovl_status ovl_deflation_info(const ovl_ctx *ctx, int *k, double *lambda, double *lambda_next, double *setup_s,
                              double *resid_max, long *matvecs);

/* Restarted Krylov sign function totals since ovl_create: cycles and products with Q^2
 * (nullable outputs). Zero while params.sign_method is OVL_SIGN_ZOLOTAREV. */
ovl_status ovl_krylov_sign_info(const ovl_ctx *ctx, long *cycles, long *matvecs);

/* Host utility: eigenvalues w[n] (ascending) and eigenvectors Z (n x n complex, row-major,
 * column j for w[j]) of the n x n complex Hermitian matrix A (row-major, interleaved re/im,
 * 2 n^2 doubles; not modified), by Householder reduction to real tridiagonal form and
 * implicit symmetric QR steps with Wilkinson shifts (Golub and Van Loan, Sec. 8.3). The
 * library uses it for the Rayleigh-Ritz steps of the low-mode eigensolver and of the
 * Krylov sign function (an implementation choice; the paper computes its eigenpairs with
 * PARPACK). OVL_EINVAL for n < 1 or NULL pointers, OVL_ENOCONV if the QR iteration takes
 * more than 60 n + 100 steps. */
ovl_status ovl_hermitian_eig(int n, const double *A, double *w, double *Z);

/* Threads per block site chosen for the FP32 Schwarz block solves of the Wilson
 * preconditioner (Sec. 5.1 smoother; an implementation choice, the paper has no
 * counterpart) and the measured time of one Schwarz cycle per variant (ms[3]: 1, 2, 4
 * threads per site; zeros when not tuned). tps, ms nullable. */
ovl_status ovl_tuning_sap(const ovl_ctx *ctx, int *tps, float *ms);

/* out_k = D_W(m0) in_k for k < n_rhs (n_rhs vectors back to back), with the multi-RHS
 * stencil: blocks of up to 12 right-hand sides per launch share every link load. */
ovl_status wilson_apply_n(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double m0);

/* out_k ~= D_N in_k for k < n_rhs (Eq. overlap_def), all right-hand sides of a block of up
 * to 12 evaluated by one lock-step FP64 multishift CG on the multi-RHS stencil; sign accuracy
 * tol for each. With deflation or the Krylov sign the right-hand sides run one at a time. */
ovl_status ovl_apply_n(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double tol);

/* out ~= sign(Q) in, Q = Gamma5 D_W(m0_ker), to relative accuracy tol (>= 1e-14), in FP64:
 * Zolotarev rational approximation + multishift CG (Sec. 2, Eq. overlap_def), or the
 * restarted Krylov method of Sec. 5.2 when params.sign_method = OVL_SIGN_KRYLOV. The
 * multishift stops when its error bound over [lambda_min, lambda_max] is below tol ||in||
 * (with the Zolotarev degree chosen so that its uniform error is <= tol / 10).
 * OVL_ENOCONV if the multishift reached params.max_ms_iter: out then holds the result formed
 * from the last iterate. OVL_EBREAKDOWN if a CG scalar became zero or non-finite (for
 * instance ||in||^2 overflowing FP64); out is then unspecified. (sign_apply_arith and
 * ovl_apply behave the same way.) */
ovl_status sign_apply(ovl_ctx *ctx, double *out, const double *in, double tol);

/* out ~= D_N in = rho in + Gamma5 sign(Q) in (Eq. overlap_def), sign to accuracy tol. */
ovl_status ovl_apply(ovl_ctx *ctx, double *out, const double *in, double tol);

/* Solves D_N x = b (Eq. linsys) for n_rhs right-hand sides to relative residual tol
 * (0 = params.tol_outer). x: n_rhs vectors; on entry the initial guess (zeros for none),
 * on exit the solutions. The method is chosen by params.precond / params.precision.
 * Returns OVL_ENOCONV if some right-hand side misses tol within max_iter (x then holds
 * the best iterate). stats may be NULL. */
ovl_status ovl_solve(ovl_ctx *ctx, double *x, const double *b, int n_rhs, double tol,
                     ovl_stats *stats);

/* Spectral data of the context: lambda_min, lambda_max of |Q|, Zolotarev error bound
 * delta on that interval, rho, m0_ker, m0_prec, sigma_min estimate. Any pointer may be NULL. */
ovl_status ovl_info(const ovl_ctx *ctx, double *lambda_min, double *lambda_max, double *delta,
                    double *rho, double *m0_ker, double *m0_prec, double *sigma_min);

/* Zolotarev coefficients on [k, 1] scaled by lambda_min (host computation, FP64):
 * sign(x) ~= d0 x (1 + sum_l a[l] / (x^2 + c[l])), x in [1, 1/k]; n poles.
 * Writes d0, a[n], c[n] and the uniform error bound delta. */
ovl_status ovl_zolotarev(double k, int n, double *d0, double *a, double *c, double *delta);

/* Instrumentation of the running library (used by the benchmark; not part of the
 * paper's method). With profiling enabled, the multishift CG records CUDA events around
 * the three kernels of one iteration of every queued chunk of check_every iterations
 * (the middle one; event nodes inside the captured graphs), a sample that keeps the
 * event nodes from slowing the other iterations, and logs the shifts each iteration
 * updated, so that algorithmic bytes (reals per site: Q p 96, residual update 144, shift
 * update 72 + 48 per updated shift) are known for every launch. The achieved rate of a
 * class is timed_bytes / ms (or timed flops / ms); its total time is estimated as
 * ms / timed * launches. */
typedef struct {
    double ms;              /* summed event time of the timed launches of the class */
    long launches;          /* all launches of the class */
    double bytes;           /* algorithmic bytes of all launches */
    double flops;           /* algorithmic flops of all launches (stencils: 1368 per site) */
    long timed;             /* launches that were timed */
    double timed_bytes;     /* algorithmic bytes of the timed launches */
} ovl_prof_kernel;

typedef struct {
    long launches;          /* kernels launched by the library since the last reset (all contexts) */
    ovl_prof_kernel k[6];   /* 0: FP64 multishift stencils, 1: FP64 shift updates,
                               2: FP32 multishift stencils, 3: FP32 shift updates,
                               4: float-float multishift stencils, 5: float-float shift updates */
    int valid;              /* 1 if every event timing could be read */
} ovl_prof;

/* Times reps back-to-back full-lattice Wilson stencil launches (out = D_W(m0_ker) in on
 * internal buffers filled with seeded pseudo-random values, after 3 untimed launches) with
 * CUDA events on the context's stream; precision 0 = FP64, 1 = FP32, 2 = float-float, 3 = FP16
 * (links and spinors, per-site spinor scale; 200 algorithmic bytes per site), 4 = BF16 (192 B).
 * *ms = average milliseconds per launch. Algorithmic traffic of one launch: 96 reals per site
 * (4 links x 12, the input and the output spinor). */
ovl_status ovl_dslash_time(ovl_ctx *ctx, int precision, int reps, double *ms);

/* As ovl_dslash_time for the multi-RHS stencil applied to nrhs (1..12) right-hand sides per
 * launch (precision 0 = FP64, 1 = FP32); *ms per launch (nrhs full-lattice applications). */
ovl_status ovl_dslash_time_n(ovl_ctx *ctx, int precision, int nrhs, int reps, double *ms);

/* Measured fused multiply-add throughput of the current device in GFLOP/s (2 flops per FMA):
 * precision 0 = FP64, 1 = FP32. Each thread runs independent FMA chains, 8 blocks of 256
 * threads per SM, one launch of >= 20 ms timed with CUDA events after a warm-up launch. It is
 * the ALU roofline denominator of the FP64 stencils (FP64) and of the float-float ones (FP32);
 * instrumentation, not part of the paper's method. Allocates 16 bytes and one stream. */
ovl_status ovl_fma_peak(int precision, double *gflops);

/* on = 1 enables event timing (allocates a small history buffer), 0 disables it. */
ovl_status ovl_prof_enable(ovl_ctx *ctx, int on);
/* Reads the accumulated counters; reset = 1 zeroes them afterwards. */
ovl_status ovl_prof_get(ovl_ctx *ctx, ovl_prof *out, int reset);

/* ---------------------------------------------------------------------------------
 * Operators in a chosen arithmetic. The paper runs its preconditioner in single precision
 * and the outer D_N products in double precision (Sec. 5.2, Sec. 5.3 and Table 3); these
 * entry points apply the same operators as wilson_apply, wilson_apply_n and sign_apply in
 * each arithmetic the solver uses (ovl_arith), so that every one of them can be checked
 * against an FP64 reference on its own. Vectors are FP64 at the boundary (layout above);
 * they are rounded to the requested arithmetic on entry and the result is returned in
 * FP64. OVL_EINVAL for an arithmetic the operator does not have.
 * --------------------------------------------------------------------------------- */

/* out = D_W(m0) in (Eq. Wilson-Dirac) in any ovl_arith, with the context's stencil variant
 * (params.stencil_tps for FP64 and FP32; float-float and 16-bit always 1 thread per site). The
 * 16-bit stencil reads 200 B per site in FP16 (192 B in BF16) against 384 B in FP32. */
ovl_status wilson_apply_arith(ovl_ctx *ctx, double *out, const double *in, double m0, int arith);

/* out_k = D_W(m0) in_k for k < n_rhs with the multi-RHS stencil (blocks of up to 12 right-hand
 * sides per launch) in arith = OVL_ARITH_FP64 or OVL_ARITH_FP32. */
ovl_status wilson_apply_n_arith(ovl_ctx *ctx, double *out, const double *in, int n_rhs, double m0, int arith);

/* out ~= sign(Q) in to relative accuracy tol (Zolotarev + multishift CG, as sign_apply) in any
 * ovl_arith. The accuracy each arithmetic can reach bounds the useful tol: float-float and FP64
 * about 1e-12, FP32 about 1e-6, FP16-stored directions about 1e-3, BF16-stored about 1e-2 (the
 * outer solver hands each arithmetic only requests above these floors). */
ovl_status sign_apply_arith(ovl_ctx *ctx, double *out, const double *in, double tol, int arith);

/* ---------------------------------------------------------------------------------
 * Two-level multigrid for D_W (the Wilson solver of the paper's preconditioner, Sec. 5.1 and
 * Table 2: two levels, red-black Schwarz smoother, adaptive setup of restriction and
 * prolongation, GMRES on the coarse level). Aggregates are the params.sap_block blocks, each
 * split by chirality (spins 0,1 and 2,3); P holds on every aggregate an orthonormal basis of
 * the test vectors; D_c = P^H D_W P couples a block to itself and its eight neighbours.
 * --------------------------------------------------------------------------------- */

/* Builds the multigrid for D_W(m0). start: n_start vectors in the boundary layout (host or
 * device) used as the initial test vectors; NULL = params.mg_nv seeded pseudo-random vectors.
 * Each is smoothed params.mg_setup_iters times by v <- v - M_SAP D_W v, then orthonormalised on
 * every aggregate. The setup is kept until the next call (or a solve that needs another m0).
 * OVL_EINVAL for n_start outside [1, 24] or blocks that leave fewer than two per direction;
 * OVL_EBREAKDOWN if a diagonal block of D_c is singular. */
ovl_status ovl_mg_setup(ovl_ctx *ctx, double m0, const double *start, int n_start);

/* out = M_MG in: one application of the two-level preconditioner for D_W(m0), FP32 inside:
 * x = P x_c with x_c from params.mg_coarse_steps steps of GMRES on D_c x_c = P^H in (right-
 * preconditioned by the inverses of D_c's diagonal blocks, stopping at relative residual
 * params.mg_coarse_tol), then x += M_SAP (in - D_W x). Makes the setup first if there is none
 * for this m0. */
ovl_status wilson_mg_apply(ovl_ctx *ctx, double *out, const double *in, double m0);

/* State of the on-the-fly preconditioner mass (params.m0_adapt): the candidate masses cand[5],
 * their scores (credited residual drop per second; 0 before use) eff[5], the number of
 * preconditioner applications made so far, and the best candidate (NaN before any score).
 * Nullable outputs. */
ovl_status ovl_m0_adapt_info(const ovl_ctx *ctx, double *cand, double *eff, long *uses, double *best);

/* Multigrid state: test vectors, coarse sites, GMRES steps of the last coarse solve, setup
 * seconds (zeros before the first setup). Nullable outputs. */
ovl_status ovl_mg_info(const ovl_ctx *ctx, int *nv, int *coarse_sites, int *last_coarse_steps, double *setup_s);

/* out = D_W(m0) in, the Wilson-Dirac operator of Eq. (Wilson-Dirac), for callers that cannot
 * allocate device memory. The paper has no counterpart to this entry point; it exists for
 * runtimes that own all device memory through their own pool, and for service loops that
 * must not call cudaMalloc/cudaFree (cudaFree synchronises the whole device). It needs no
 * context (ovl_create allocates) and calls no allocating routine.
 * out, in: V*12 complex doubles, gauge: V*4*9 complex doubles, all DEVICE memory in the
 * boundary layout above; dims as for ovl_create; antiperiodic: 1 = antiperiodic time boundary.
 * All nine complex entries of every link are used as given; unlike ovl_create, no SU(3)
 * check is made. The three pointers must be memory of the current device (or managed
 * memory); pointers into another GPU are rejected with OVL_EINVAL. The library cannot see
 * buffer sizes: out and in must hold V*12 and gauge V*4*9 complex doubles.
 * Working memory: one fixed device array inside the library of 16384 lattice sites
 * (about 15.7 MB), reserved on every GPU that loads the library until the process exits;
 * larger lattices are rejected with OVL_EINVAL. The first call on a device looks the
 * array's address up on that device (make this first call before any stream capture) and
 * keeps it for the life of the process: it belongs to the device's primary context, so
 * after cudaDeviceReset, or with another driver context current, the kept address is stale
 * and this entry point must not be called again in that process.
 * All calls share the array: calls whose work overlaps on the GPU (other streams, other
 * host threads) race and give undefined results; calls ordered on one stream are safe.
 * The work is enqueued on cuda_stream (NULL = the legacy default stream) and the call
 * returns without waiting: out is ready once that stream has finished it. Errors are
 * reported by the return status, with the reason in ovl_last_error(NULL). */
ovl_status wilson_apply_noalloc(double *out, const double *in, const double *gauge, const int dims[4],
                                double m0, int antiperiodic, void *cuda_stream);

/* ---------------------------------------------------------------------------------
 * Serving: overlap solves submitted as they arrive, run concurrently on the current GPU.
 * (Not part of the paper's method; a service layer around ovl_create/ovl_solve.)
 * `slots` worker threads run requests concurrently; every context issues its work on a CUDA
 * stream of its own, so the kernels of concurrent requests overlap on the device. A queued request starts as soon as a slot is
 * free and its estimated device memory fits hbm_budget next to the running requests and
 * the cached contexts (first fit in arrival order). After a request completes its context
 * (gauge field, spectral interval, coefficients, workspaces) stays resident, keyed by
 * gauge_key and the operator parameters, and later requests with the same key reuse it;
 * idle contexts are evicted least recently used first when memory is needed.
 * --------------------------------------------------------------------------------- */
typedef struct ovl_server ovl_server;

typedef struct {
    const double *gauge;        /* V*4*9 complex doubles (host or device), as for ovl_create */
    long gauge_key;             /* nonzero: reuse resident contexts of equal key and operator */
    int dims[4];
    double rho, mu;
    int n_rhs;
    const double *b;            /* n_rhs right-hand sides (host or device) */
    double *x;                  /* n_rhs initial guesses in, solutions out */
    double tol;                 /* 0 = params.tol_outer */
    const ovl_params *params;   /* NULL = defaults; copied at submission */
} ovl_request;

typedef struct {
    int done;                   /* 1 once finished (successfully or not) */
    ovl_status status;
    ovl_stats stats;
    double queue_s;             /* submission -> start */
    double run_s;               /* start -> completion */
    double latency_s;           /* submission -> completion */
    size_t device_bytes;        /* device memory the request held */
    char message[160];          /* error text when status != OVL_OK */
} ovl_result;

/* slots: concurrent requests (1..64); hbm_budget: bytes of device memory the server may use
 * (0 = 90% of the free memory at creation). */
ovl_status ovl_server_create(ovl_server **srv, int slots, size_t hbm_budget);
/* Host only (no device call): the device memory the server reserves for req at admission,
 * an upper estimate of what ovl_create and ovl_solve allocate for its lattice, precision,
 * preconditioner, sign method, deflation and right-hand sides (params NULL = defaults).
 * OVL_EINVAL for NULL pointers, n_rhs < 1 or a non-positive extent. */
ovl_status ovl_request_bytes(const ovl_request *req, size_t *bytes);
/* Queues a request and returns its ticket. The buffers it points to (gauge, b, x) must stay
 * valid until the request is done. OVL_ENOMEM: the request can never fit the budget. */
ovl_status ovl_server_submit(ovl_server *srv, const ovl_request *req, long *ticket);
/* Non-blocking status of a ticket (res->done == 0 while queued or running). */
ovl_status ovl_server_query(ovl_server *srv, long ticket, ovl_result *res);
/* Blocks until the ticket's request is done; res may be NULL. */
ovl_status ovl_server_wait(ovl_server *srv, long ticket, ovl_result *res);
/* Latency percentiles (s) over completed requests, completed requests per second of wall time
 * (first submission to last completion), reserved-memory high-water mark. Nullable outputs. */
ovl_status ovl_server_report(ovl_server *srv, double *p50, double *p99, double *solves_per_s,
                             size_t *hbm_high_water, long *completed, long *failed);
/* Finishes the queued requests, stops the workers and frees every resident context. */
ovl_status ovl_server_destroy(ovl_server *srv);

/* Destroys the context and frees its device memory. NULL is a no-op. */
ovl_status ovl_destroy(ovl_ctx *ctx);

/* One-line description of the last error on ctx (or of the last failed
 * ovl_create on this thread when ctx is NULL). Never NULL. */
const char *ovl_last_error(const ovl_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* OVL_H */

// Two-level aggregation multigrid for D_W (internal interface): the Wilson solver of the
// paper's preconditioner (Sec. 5.1, Table 2: DD-alpha-AMG with two levels, a red-black
// Schwarz smoother, an adaptive setup and GMRES on the coarse level).
//
// Aggregates are the Schwarz blocks split by chirality (spins {0,1} and {2,3}); a coarse
// site is a block, with nc = 2 nv coarse dofs ordered (chirality, test vector). Coarse
// vectors are float2 [Nb][nc]. The coarse operator couples a block to itself and its eight
// neighbour blocks: D_c[b][d] is an nc x nc matrix for d = 0 (self), 1 + 2 mu (block
// b + mu) and 2 + 2 mu (block b - mu), stored column-major ([b][d][col][row]).
#pragma once
#include "internal.h"
#include "sap.h"

namespace ovl {

constexpr int kMgMaxNv = 24;        // test vectors (nc = 2 nv <= 48)
constexpr int kMgMaxSteps = 64;     // coarse GMRES steps per solve

// Device scalars of one coarse GMRES solve (right-preconditioned by the block inverses).
struct MgCoarseState {
    int m;                  // steps of this solve
    int j;                  // current step
    int done;               // 1: converged or m steps done (kernels then do nothing)
    int steps;              // steps taken
    double tol;             // stop when the residual estimate <= tol * beta0
    double beta0;
    float scale;            // 1 / norm of the vector that becomes v_j
    double H[(kMgMaxSteps + 1) * kMgMaxSteps * 2];   // Hessenberg, complex, H(i, j) at [(j*(kMgMaxSteps+1)+i)*2]
    double g[(kMgMaxSteps + 1) * 2];                 // rotated right-hand side, complex
    double cs[kMgMaxSteps];                          // Givens cosines (real)
    double sn[kMgMaxSteps * 2];                      // Givens sines (complex)
    double y[kMgMaxSteps * 2];                       // least-squares solution
};

struct MgData {
    int nv = 0, nc = 0, nb = 0;     // test vectors, coarse dofs per site, coarse sites (blocks)
    long ncv = 0;                   // coarse vector length nb * nc
    float4 *P = nullptr;            // nv FP32 even-odd spinors, orthonormal on every aggregate
    float2 *Dc = nullptr;           // coarse operator [nb][9][nc][nc]
    float2 *A = nullptr;            // D_c M^{-1}, same layout (the right-preconditioned operator)
    float2 *Minv = nullptr;         // inverses of the self blocks [nb][nc][nc]
    int *nbr = nullptr;             // [nb][9] coarse neighbour of each direction
    float2 *V = nullptr;            // coarse GMRES basis (kMgMaxSteps + 1) x ncv
    float2 *w[2] = {nullptr, nullptr};   // coarse work vectors (alternating)
    float2 *rc = nullptr, *xc = nullptr; // coarse right-hand side and solution
    double *part = nullptr;         // per-block partial sums [kMgMaxSteps + 2][nb]
    unsigned *counter = nullptr;    // last-block counter
    MgCoarseState *cs = nullptr;
    float4 *t1 = nullptr, *t2 = nullptr, *t3 = nullptr;   // fine FP32 scratch spinors
    float4 *tin = nullptr, *tout = nullptr;               // fixed input / output of the captured application
    cudaGraphExec_t graph = nullptr;   // one application captured as a CUDA graph (rebuilt with the setup)
    long graph_launches = 0;           // kernels in that graph
    double m0 = 0;                  // mass the setup was made for
    bool ready = false;
    double setup_s = 0;
    long coarse_steps = 0;          // coarse GMRES steps since the setup
    long applications = 0;
};

// r_c = P^H r (restriction); out[b * ob + off + row], row = chi * nv + k
cudaError_t mg_restrict(const Geom &g, const SapGeom &sg, const float4 *P, int nv, const float4 *r, float2 *out,
                        long ob, long off, cudaStream_t st);
// out (+)= P x_c (prolongation; add = accumulate into out)
cudaError_t mg_prolong(const Geom &g, const SapGeom &sg, const float4 *P, int nv, const float2 *xc, float4 *out,
                       bool add, cudaStream_t st);
// out = part of D_W(m0) in: part 0 = (m0 + 4) in + the hops inside the block, part 1 + 2 mu
// (2 + 2 mu) = the forward (backward) hops in direction mu that cross a block face
cudaError_t mg_dpart(const Geom &g, const SapGeom &sg, const float4 *U, const float4 *in, float4 *out, float m0,
                     int part, cudaStream_t st);
// out = v with the components of chirality 1 - chi zeroed
cudaError_t mg_chiral_mask(const Geom &g, const float4 *v, float4 *out, int chi, cudaStream_t st);
// orthonormalise the nv vectors on every aggregate (block Gram-Schmidt, two passes)
cudaError_t mg_orthonormalise(const Geom &g, const SapGeom &sg, float4 *P, int nv, cudaStream_t st);
// A[b][d] = Dc[b][d] Minv[nbr[b][d]]
cudaError_t mg_right_precondition(const MgData &mg, cudaStream_t st);
// x_c ~ D_c^{-1} r_c: m steps of right-preconditioned GMRES from 0, stopping once the
// residual estimate is <= tol ||r_c||; the kernels read their step count from the device
cudaError_t mg_coarse_solve(const MgData &mg, int m, double tol, cudaStream_t st);
// y = D_c x (coarse operator applied; for tests)
cudaError_t mg_coarse_apply(const MgData &mg, const float2 *x, float2 *y, cudaStream_t st);

}  // namespace ovl

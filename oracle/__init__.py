"""CPU FP64 oracle for the overlap-operator hot path — TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package. The library's product path never imports it, and it imports nothing
from the library. It is a plain, slow, checkable restatement of what the
paper defines:

  * gamma.py       gamma matrices (Eq. commutativity_rel, gamma_5 of Sec. 2)
  * dense.py       dense D_W (Eq. Wilson-Dirac), Q = Gamma5 D_W, sign(Q) by a
                   Hermitian eigendecomposition (Lemma svd_kernel), D_N
                   (Eq. overlap_def), dense LU solve of D_N psi = eta (Eq. linsys)
  * observables.py plaquettes (Eqs. plaquette_def1/2), Wilson action, the
                   non-normality measure of Prop. Fnorm
  * zolotarev.py   Zolotarev's optimal rational approximation of sign(x)
                   (not in the paper, which uses a thick-restart Krylov
                   method; Zolotarev's form is the one the GPU path evaluates)
  * sparse.c/.py   definitional D_W stencil with full 3x3 links in plain C,
                   and sign(Q) by one plain CG per Zolotarev pole
  * solvers.py     textbook restarted GMRES(m) and right-preconditioned
                   FGMRES(m) (Sec. 5.1)
  * krylov_sign.py the restarted Krylov sign function of Sec. 5.2
                   (quadrature-based restarts, optional thick restarts)
  * sap.py         red-black multiplicative Schwarz with minimal-residual
                   block solves (the Wilson preconditioner's smoother, Sec. 5.1)

Every function is pinned by tests against closed forms, invariants or
library routines (free-field spectrum, Gamma5-hermiticity, sign^2 = I,
Ginsparg-Wilson, normality, gauge covariance, Prop. Fnorm, the alternation
theorem for the Zolotarev coefficients, an SVD polar factor for sign(Q), the
closed form of restarted Arnoldi for matrix functions, block Gauss-Seidel
for one Schwarz cycle with exact block solves).
"""

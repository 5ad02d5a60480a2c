"""Restarted Krylov approximation of sign(Q) b with thick restarts (Sec. 5.2) — oracle.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg call this module; the library never does.

Sec. 5.2 approximates sign(Gamma5 D_W) chi by a restarted Krylov subspace
method for matrix functions that allows thick restarts (the quadrature-based
restarts of Frommer, Guettel and Schweitzer, SIAM J. Matrix Anal. Appl. 35,
2014). For a Hermitian, nonsingular Q the method is stated here as follows.

  sign(Q) b = f(A) c   with A = Q^2 (Hermitian positive definite), c = Q b,
                       f(z) = z^{-1/2} = (2/pi) int_0^inf ds / (z + s^2).

  Quadrature. With s = e^u the integrand e^u / (z + e^{2u}) decays like
  e^{-|u|} in both directions and is analytic in the strip |Im u| < pi/2, so
  the trapezoidal rule in u converges geometrically:
      f(z) ~ r(z) = sum_j w_j / (z + t_j),  t_j = e^{2 u_j},  w_j = (2/pi) h e^{u_j},
  u_j = u_lo + j h. The truncation u_lo = ln(a_lo)/2 - 37, u_hi = ln(a_hi)/2 + 37
  (a_lo <= spectrum of A <= a_hi) leaves tails below e^{-37} of f, and h = 0.2
  puts the discretisation error near exp(-pi^2 / h) ~ 4e-22.

  Cycle k works on an orthonormal basis W = [w_0 .. w_{m-1}] with
      A W = W H + beta w_m e_{m-1}^T,   H = W^H A W   (m x m, Hermitian),
  and a start column s: W e_s is the vector v the previous cycle's error is
  collinear with (s = 0 and v = c / ||c|| in cycle 1). The error of the
  current approximation f_{k-1} is
      f(A) c - f_{k-1} = sum_j w_j xi_j (A + t_j)^{-1} v      (xi_j = ||c|| at k = 1).
  Galerkin step for every shifted system: y_j = (H + t_j)^{-1} e_s, and
      f_k = f_{k-1} + W sum_j w_j xi_j y_j.
  Its residual is (A + t_j)(W y_j) - v = beta (e_{m-1}^T y_j) w_m, hence the
  new error is sum_j w_j xi_j' (A + t_j)^{-1} w_m with
      xi_j' = -xi_j beta (e_{m-1}^T y_j),     v' = w_m.
  Since ||(A + t)^{-1}|| <= 1 / (a_lo + t), the error is at most
      bound_k = sum_j w_j |xi_j'| / (a_lo + t_j);
  the iteration stops when bound_k <= tol ||b|| (||sign(Q) b|| = ||b||).

  Restart. Without thick restart (keep = 0) the next basis starts at w_m
  (s = 0). With thick restart the eigenpairs (theta_i, S e_i) of H of the
  `keep` smallest Ritz values are kept: W' = [W S_keep, w_m], s = keep, and
  A (W S e_i) = theta_i W S e_i + beta (e_{m-1}^T S e_i) w_m gives the new
  projected matrix diag(theta) bordered by beta S_{m-1,i} in row and
  column `keep`. The basis is then extended by Lanczos steps with two-pass
  classical Gram-Schmidt against all columns (Eiermann, Ernst and Guettel,
  SIAM J. Matrix Anal. Appl. 32, 2011, for deflated restarts of f(A) b).
"""

import numpy as np

QUAD_H = 0.2
QUAD_TAIL = 37.0


def quadrature(a_lo, a_hi, h=QUAD_H, tail=QUAD_TAIL):
    """Nodes t_j and weights w_j of r(z) = sum w_j / (z + t_j) ~ z^{-1/2} on [a_lo, a_hi]."""
    u_lo = 0.5 * np.log(a_lo) - tail
    u_hi = 0.5 * np.log(a_hi) + tail
    n = int(np.ceil((u_hi - u_lo) / h)) + 1
    u = u_lo + h * np.arange(n)
    return np.exp(2.0 * u), (2.0 / np.pi) * h * np.exp(u)


def _extend(matvec, W, H, j0, m):
    """Lanczos steps j0..m-1 with two-pass classical Gram-Schmidt: fills W[:, j0+1..m],
    column j of H on and above the diagonal with the Gram-Schmidt coefficients and
    H[j+1, j] with the new norm (the caller takes the Hermitian part); returns
    (beta, m_eff) with m_eff < m on an exact invariant subspace."""
    beta = 0.0
    for j in range(j0, m):
        w = matvec(W[:, j])
        for _ in range(2):
            h = W[:, :j + 1].conj().T @ w
            H[:j + 1, j] += h
            w = w - W[:, :j + 1] @ h
        beta = np.linalg.norm(w)
        if beta <= 1e-14 * max(np.abs(H[:j + 1, :j + 1]).max(), 1e-300):
            return 0.0, j + 1
        W[:, j + 1] = w / beta
        if j + 1 < m:
            H[j + 1, j] = beta
    return beta, m


def krylov_sign(q_apply, b, a_lo, a_hi, tol, m=40, keep=0, max_cycles=500, history=False):
    """sign(Q) b for Hermitian Q given by q_apply(v) = Q v (flat complex vectors).

    a_lo, a_hi: bounds of the spectrum of A = Q^2. Returns (x, info) with info =
    {"converged", "cycles", "matvecs" (products with A), "bounds" (error bound after each
    cycle)}; with history=True also "cycle_data": per cycle (W[:, :m], H, beta, s, f_k).
    After max_cycles without reaching tol, x is the last iterate and converged is False.
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    n = b.size
    bnorm = np.linalg.norm(b)
    info = {"converged": True, "cycles": 0, "matvecs": 0, "bounds": [], "cycle_data": []}
    if bnorm == 0.0:
        return np.zeros(n, dtype=np.complex128), info
    t, w = quadrature(a_lo, a_hi)
    c = q_apply(b)
    cnorm = np.linalg.norm(c)
    xi = np.full(t.size, cnorm, dtype=np.complex128)
    f = np.zeros(n, dtype=np.complex128)
    W = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m, m), dtype=np.complex128)
    W[:, 0] = c / cnorm
    j0, s = 0, 0

    def a_apply(v):
        info["matvecs"] += 1
        return q_apply(q_apply(v))

    for cycle in range(max_cycles):
        beta, me = _extend(a_apply, W, H, j0, m)
        Hm = 0.5 * (H[:me, :me] + H[:me, :me].conj().T)
        theta, S = np.linalg.eigh(Hm)
        # y_j = S (theta + t_j)^{-1} S^H e_s for every node; the update is W sum_j w_j xi_j y_j
        q = S[s, :].conj()                                  # S^H e_s
        D = q[None, :] / (theta[None, :] + t[:, None])      # [node, eigen] coefficients of S
        coef = S @ ((w * xi) @ D)
        f = f + W[:, :me] @ coef
        info["cycles"] = cycle + 1
        gam = D @ S[me - 1, :]                              # e_{m-1}^T y_j
        xi = -xi * beta * gam
        bound = float(np.sum(w * np.abs(xi) / (a_lo + t)))
        info["bounds"].append(bound)
        if history:
            info["cycle_data"].append((W[:, :me].copy(), Hm.copy(), beta, s, f.copy()))
        if beta == 0.0 or bound <= tol * bnorm:
            return f, info
        # restart: keep the Ritz vectors of the `keep` smallest Ritz values, then w_m
        kk = min(keep, me - 1)
        last = W[:, me].copy()
        if kk > 0:
            W[:, :kk] = W[:, :me] @ S[:, :kk]
        W[:, kk] = last
        H[:] = 0.0
        for i in range(kk):
            H[i, i] = theta[i]
            H[kk, i] = beta * S[me - 1, i]   # column kk above the diagonal comes from Gram-Schmidt
        j0, s = kk, kk
    info["converged"] = False
    return f, info

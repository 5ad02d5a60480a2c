"""Textbook restarted GMRES(m) / right-preconditioned FGMRES(m) (Sec. 5.1).

Sec. 5.1 solves D_N psi = eta with GMRES(100), and with FGMRES(100) when the
(non-stationary) Wilson-Dirac preconditioner is applied from the right. This
is the plain algorithm (Saad, Iterative Methods for Sparse Linear Systems):
Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
matrix, x += Z y at the end of a cycle (Z = V for GMRES), restart from the
true residual. Stopping rule: ||b - A x|| <= tol ||b|| (Sec. 5.1, "reduce the
initial residual by a factor of 1e-8" with x0 = 0).
"""

import numpy as np


def fgmres(matvec, b, tol, restart=100, maxiter=100000, x0=None, precond=None):
    """Solve A x = b. precond(v) ~ A^{-1} v is applied from the right (flexible).

    Returns (x, info) with info = {"iters", "converged", "history"}; history
    holds the Arnoldi residual estimate after every iteration.
    """
    b = np.asarray(b, dtype=np.complex128)
    shape = b.shape
    bv = b.reshape(-1)
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    bnorm = np.linalg.norm(bv)
    hist = []
    if bnorm == 0.0:
        return np.zeros(shape, dtype=np.complex128), {"iters": 0, "converged": True, "history": hist}
    its = 0
    while its < maxiter:
        r = bv - matvec(x.reshape(shape)).reshape(-1)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            return x.reshape(shape), {"iters": its, "converged": True, "history": hist}
        m = restart
        Vb = np.zeros((m + 1, bv.size), dtype=np.complex128)
        Zb = np.zeros((m, bv.size), dtype=np.complex128) if precond is not None else None
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        j_done = 0
        for j in range(m):
            z = Vb[j] if precond is None else precond(Vb[j].reshape(shape)).reshape(-1)
            if precond is not None:
                Zb[j] = z
            w = matvec(z.reshape(shape)).reshape(-1)
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                Vb[j + 1] = w / H[j + 1, j]
            # rotation i maps (h_i, h_{i+1}) -> (conj(c) h_i + conj(s) h_{i+1}, -s h_i + c h_{i+1})
            for i in range(j):                        # previous rotations
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]               # new rotation zeroing H[j+1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = bb / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or its >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        basis = Vb[:j_done] if precond is None else Zb[:j_done]
        x = x + basis.T @ y
    r = bv - matvec(x.reshape(shape)).reshape(-1)
    return x.reshape(shape), {"iters": its, "converged": np.linalg.norm(r) <= tol * bnorm,
                              "history": hist}


def power_iteration_max_real(matvec, v0, iters):
    """Rough largest-real-part eigenvalue estimate of a non-Hermitian operator.

    Sec. 5.1 obtains sigma~_max by a fixed number of power iterations; the
    Rayleigh quotient v^H A v of the normalised iterate gives its real part.
    """
    v = np.asarray(v0, dtype=np.complex128)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = matvec(v)
        lam = np.vdot(v, w)
        v = w / np.linalg.norm(w)
    return float(np.real(lam))

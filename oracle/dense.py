"""Dense / sparse-matrix FP64 oracle of the overlap operator (Secs. 2, 3, 5).

Component index of a spinor: 12*s + 3*spin + colour, s the lexicographic site
index ((x0*L1 + x1)*L2 + x2)*L3 + x3.

  wilson_matrix      D_W(m0) entrywise from Eq. (Wilson-Dirac) with a = 1
  gamma5_matrix      Gamma5 = I_V (x) gamma_5 (x) I_3 (Sec. 2)
  sign_hermitian     sign(Q) = W sign(Delta) W^H (Lemma svd_kernel, proof)
  overlap_dense      D_N = rho I + Gamma5 sign(Gamma5 D_W(m0_ker)) (Eq. overlap_def)
  rho_from_mu        rho = (-mu/2 + m0_ker) / (mu/2 + m0_ker) (Sec. 5)
  default_prec_mass  m0^def = omega^def rho + m0_ker, omega^def = -m0_ker - sigma_min
                     (Eq. default_m)

Boundary conditions: periodic in all directions, optionally antiperiodic in
the time direction x0: a hop that crosses the x0 boundary carries a factor -1.
"""

import numpy as np
import scipy.sparse as sp

from .gamma import GAMMA, GAMMA5, I4


def coords(dims):
    """[V,4] integer coordinates in lexicographic order (x3 fastest)."""
    g = np.meshgrid(*[np.arange(L) for L in dims], indexing="ij")
    return np.stack([a.reshape(-1) for a in g], axis=1)


def lex(x, dims):
    x0, x1, x2, x3 = (x[..., i] % dims[i] for i in range(4))
    return ((x0 * dims[1] + x1) * dims[2] + x2) * dims[3] + x3


def wilson_matrix(U, dims, m0, antiperiodic=True):
    """Sparse 12V x 12V D_W(m0) of Eq. (Wilson-Dirac), a = 1.

    (D_W psi)(x) = (m0+4) psi(x)
                   - 1/2 sum_mu (I - gamma_mu) (x) U_mu(x)       psi(x+mu)
                   - 1/2 sum_mu (I + gamma_mu) (x) U_mu(x-mu)^H  psi(x-mu)
    """
    dims = tuple(dims)
    V = int(np.prod(dims))
    X = coords(dims)
    s = lex(X, dims)
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")
    for mu in range(4):
        e = np.zeros(4, dtype=int)
        e[mu] = 1
        sf = lex(X + e, dims)
        sb = lex(X - e, dims)
        phf = np.ones(V)
        phb = np.ones(V)
        if antiperiodic and mu == 0:
            phf[X[:, 0] == dims[0] - 1] = -1.0
            phb[X[:, 0] == 0] = -1.0
        Umu = U[:, mu]                                   # U_mu(x)
        Umu_b = U[sb, mu]                                # U_mu(x - mu)
        Kf = np.einsum("ij,sab->siajb", I4 - GAMMA[mu], Umu).reshape(V, 12, 12)
        Kb = np.einsum("ij,sab->siajb", I4 + GAMMA[mu],
                       np.conj(np.swapaxes(Umu_b, -1, -2))).reshape(V, 12, 12)
        for K, nb, ph in ((Kf, sf, phf), (Kb, sb, phb)):
            rows.append((12 * s[:, None, None] + ii[None]).reshape(-1))
            cols.append((12 * nb[:, None, None] + jj[None]).reshape(-1))
            vals.append((-0.5 * ph[:, None, None] * K).reshape(-1))
    rows.append(np.arange(12 * V))
    cols.append(np.arange(12 * V))
    vals.append(np.full(12 * V, m0 + 4.0, dtype=np.complex128))
    D = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(12 * V, 12 * V))
    return D.tocsr()


def gamma5_matrix(V):
    return sp.kron(sp.identity(V), sp.kron(sp.csr_matrix(GAMMA5), sp.identity(3))).tocsr()


def gamma5_vec(psi):
    """Gamma5 psi for psi shaped [..., V, 4, 3]."""
    return np.einsum("ij,...vjc->...vic", GAMMA5, psi)


def sign_hermitian(Q, rel_gap=1e-12):
    """sign(Q) = W sign(Delta) W^H for Hermitian Q (Lemma svd_kernel, proof).

    sign is undefined at 0 (Sec. 2); a spectrum touching 0 (relative to the
    largest |eigenvalue|) is rejected.
    """
    Q = np.asarray(Q)
    w, W = np.linalg.eigh(Q)
    aw = np.abs(w)
    if aw.min() < rel_gap * aw.max():
        raise ValueError("sign(Q) undefined: Q has an eigenvalue at 0")
    return (W * np.sign(w)[None, :]) @ W.conj().T, w


def rho_from_mu(mu, m0_ker):
    """rho = (-mu/2 + m0_ker) / (mu/2 + m0_ker) (Sec. 5)."""
    return (-mu / 2.0 + m0_ker) / (mu / 2.0 + m0_ker)


def overlap_dense(U, dims, rho, m0_ker, antiperiodic=True):
    """Dense D_N = rho I + Gamma5 sign(Gamma5 D_W(m0_ker)) (Eq. overlap_def).

    Returns (D_N, sign(Q), eigenvalues of Q).
    """
    V = int(np.prod(dims))
    Dw = wilson_matrix(U, dims, m0_ker, antiperiodic).toarray()
    G5 = gamma5_matrix(V).toarray()
    Q = G5 @ Dw
    Q = 0.5 * (Q + Q.conj().T)       # Hermitian by Eq. (gamma_5_symmetry); symmetrise rounding
    S, w = sign_hermitian(Q)
    DN = rho * np.eye(12 * V) + G5 @ S
    return DN, S, w


def overlap_solve_dense(DN, eta):
    """psi = D_N^{-1} eta by dense LU (Eq. linsys)."""
    return np.linalg.solve(DN, eta.reshape(-1)).reshape(eta.shape)


def default_prec_mass(rho, m0_ker, sigma_min):
    """m0^def of Eq. (default_m)."""
    omega = -m0_ker - sigma_min
    return omega * rho + m0_ker

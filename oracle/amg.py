"""Two-level aggregation multigrid preconditioner for D_W — oracle.

TEST INFRASTRUCTURE ONLY: the tests call this module; the library never does.

Sec. 5.1 solves the Wilson systems of its preconditioner with DD-alpha-AMG: two levels
(Table 2), a red-black multiplicative Schwarz smoother, an adaptive setup that builds the
restriction and prolongation and with them the coarse system, and GMRES on the coarse
level. The paper gives no further detail and refers to its reference. The reading used by
the library, written out plainly here:

  aggregates   the Schwarz blocks (sap.blocks), each split by chirality: spins {0, 1}
               (gamma5 = -1 in the chiral basis) and spins {2, 3} (gamma5 = +1). Aggregate
               (b, chi) holds the dofs of block b with spins of chirality chi;
  setup        n_v test vectors from given start vectors v_k: nu times
                   v_k <- v_k - M_SAP D_W v_k
               (the smoother applied to D_W x = 0); then on every aggregate the restrictions
               of v_0 .. v_{n_v - 1} are orthonormalised (any orthonormal basis of their span:
               the preconditioner depends only on the spans). Column (b, chi, k) of P is the
               k-th basis vector of aggregate (b, chi), zero elsewhere;
  coarse op    D_c = P^H D_W P, coarse vector index (b, chi, k) with k fastest, then chi;
  coarse solve one cycle of m steps of GMRES from 0 on D_c, right-preconditioned by the
               inverses of the diagonal blocks D_c[b, b] (size 2 n_v, both chiralities of
               block b), i.e. x_c = M^{-1} V_m y, y = argmin ||r_c - D_c M^{-1} V_m y||;
  application  x = P x_c with x_c the coarse solve of P^H r; then x += M_SAP (r - D_W x).
"""

import numpy as np
import scipy.sparse as sps

from . import dense, sap


def aggregates(dims, block):
    """[(b, chi, dof index array)] in the order of the coarse vector: block b (sap.blocks
    order), then chirality chi."""
    out = []
    for b, (_, dof) in enumerate(sap.blocks(dims, block)):
        spin = (dof % 12) // 3
        for chi in (0, 1):
            out.append((b, chi, dof[(spin // 2) == chi]))
    return out


def smooth_test_vectors(U, dims, m0, start, nu, block, cycles, mr_steps, antiperiodic=True):
    """v_k <- v_k - M_SAP D_W v_k, nu times, for every start vector [n_v, V, 4, 3]."""
    D = dense.wilson_matrix(U, dims, m0, antiperiodic)
    out = []
    for v0 in start:
        v = np.asarray(v0, dtype=np.complex128).reshape(-1).copy()
        for _ in range(nu):
            w = sap.sap_apply(U, dims, m0, (D @ v).reshape(np.shape(v0)), block, cycles, mr_steps, antiperiodic)
            v = v - w.reshape(-1)
        out.append(v)
    return np.stack(out, axis=1)


def prolongation(dims, block, vecs):
    """P as a sparse [12 V, n_agg n_v] matrix: per aggregate an orthonormal basis (numpy QR) of
    the restrictions of the columns of vecs [12 V, n_v]."""
    aggs = aggregates(dims, block)
    nv = vecs.shape[1]
    rows, cols, vals = [], [], []
    for a, (b, chi, idx) in enumerate(aggs):
        Q, _ = np.linalg.qr(vecs[idx])
        for k in range(nv):
            rows.append(idx)
            cols.append(np.full(idx.size, a * nv + k))
            vals.append(Q[:, k])
    N = vecs.shape[0]
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, len(aggs) * nv))


def coarse_operator(U, dims, m0, P, antiperiodic=True):
    """D_c = P^H D_W P (dense)."""
    D = dense.wilson_matrix(U, dims, m0, antiperiodic)
    return (P.conj().T @ (D @ P)).toarray()


def block_jacobi_inverse(Dc, nv):
    """Inverses of the diagonal blocks of D_c, one per lattice block (2 n_v x 2 n_v)."""
    n = Dc.shape[0] // (2 * nv)
    Minv = np.zeros_like(Dc)
    for b in range(n):
        s = slice(2 * nv * b, 2 * nv * (b + 1))
        Minv[s, s] = np.linalg.inv(Dc[s, s])
    return Minv


def gmres_steps(A, r, Minv, m):
    """One GMRES cycle of m steps from x = 0 on A x = r, right-preconditioned by Minv:
    Arnoldi (modified Gram-Schmidt) on A Minv from r / ||r||, y = argmin ||beta e_1 - H y||,
    x = Minv V y. Stops early on an exact Krylov space (breakdown)."""
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return np.zeros_like(r)
    V = [r / beta]
    H = np.zeros((m + 1, m), dtype=complex)
    k = m
    for j in range(m):
        w = A @ (Minv @ V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * beta:
            k = j + 1
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(k + 1, dtype=complex)
    e1[0] = beta
    y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
    return Minv @ (np.stack(V[:k], axis=1) @ y)


class TwoLevel:
    """The two-level preconditioner for D_W(m0) built from start vectors [n_v, V, 4, 3]."""

    def __init__(self, U, dims, m0, start, nu, block, cycles, mr_steps, coarse_steps, antiperiodic=True):
        self.U, self.dims, self.m0, self.block = U, tuple(dims), m0, tuple(block)
        self.cycles, self.mr_steps, self.ap = cycles, mr_steps, antiperiodic
        self.nv = len(start)
        self.coarse_steps = coarse_steps
        vecs = smooth_test_vectors(U, dims, m0, start, nu, block, cycles, mr_steps, antiperiodic)
        self.P = prolongation(dims, block, vecs)
        self.D = dense.wilson_matrix(U, dims, m0, antiperiodic)
        self.Dc = (self.P.conj().T @ (self.D @ self.P)).toarray()
        self.Minv = block_jacobi_inverse(self.Dc, self.nv)

    def coarse_solve(self, rc):
        if self.coarse_steps is None:          # exact coarse solve
            return np.linalg.solve(self.Dc, rc)
        return gmres_steps(self.Dc, rc, self.Minv, self.coarse_steps)

    def apply(self, r):
        """x = P x_c (x_c the coarse solve of P^H r), then x += M_SAP (r - D_W x)."""
        shape = np.shape(r)
        rr = np.asarray(r, dtype=np.complex128).reshape(-1)
        x = self.P @ self.coarse_solve(self.P.conj().T @ rr)
        res = (rr - self.D @ x).reshape(shape)
        x = x + sap.sap_apply(self.U, self.dims, self.m0, res, self.block, self.cycles, self.mr_steps,
                              self.ap).reshape(-1)
        return x.reshape(shape)

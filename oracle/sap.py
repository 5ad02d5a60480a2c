"""Red-black multiplicative Schwarz with minimal-residual block solves — oracle.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU leg call this module;
the library never does.

Sec. 5.1 preconditions with D_W(m0_prec)^{-1} applied inexactly; the smoother of its
multigrid solver is a red-black multiplicative Schwarz method whose details the paper
does not give. The reading used by the library, written out plainly here:

  blocks   the lattice is cut into blocks of b0 x b1 x b2 x b3 sites; block B has
           block coordinates (B0, B1, B2, B3) and colour (B0 + B1 + B2 + B3) mod 2;
           colour 0 ("red") is swept first;
  D_BB     D_W restricted to the sites of B: the submatrix of D_W on B, i.e. every hop
           that leaves the block is dropped (Dirichlet boundary). With at least two
           blocks in every direction no hop wraps around inside a block, so the
           submatrix is exactly that;
  cycle    for colour c in (0, 1):
               r = v - D_W x                       (x before this colour's sweep)
               for every block B of colour c:  x_B += MR_k(D_BB, r_B)
  MR_k     k minimal-residual steps from e = 0, s = r_B:
               q = D_BB s,  alpha = <q, s> / <q, q>,  e += alpha s,  s -= alpha q
           (stopping early if q = 0);
  M_SAP v  `cycles` cycles from x = 0.

Blocks of one colour share no face when every direction has an even number of
blocks; with an odd number they can touch across the periodic boundary, and the
residual r taken once per colour keeps their corrections independent in both cases.
"""

import numpy as np

from . import dense


def blocks(dims, block):
    """[(colour, dof index array)] of every block, in block-lexicographic order."""
    dims, block = tuple(dims), tuple(block)
    nblk = [dims[m] // block[m] for m in range(4)]
    if any(dims[m] % block[m] for m in range(4)) or min(nblk) < 2:
        raise ValueError("blocks must tile the lattice with at least two blocks per direction")
    X = dense.coords(dims)
    bc = X // np.asarray(block)[None, :]
    bid = ((bc[:, 0] * nblk[1] + bc[:, 1]) * nblk[2] + bc[:, 2]) * nblk[3] + bc[:, 3]
    site = np.arange(X.shape[0])
    out = []
    for b in range(int(np.prod(nblk))):
        sites = site[bid == b]
        colour = int(bc[sites[0]].sum() % 2)
        dof = (12 * sites[:, None] + np.arange(12)[None, :]).reshape(-1)
        out.append((colour, dof))
    return out


def minimal_residual(A, r, steps):
    """e ~ A^{-1} r by `steps` minimal-residual steps from e = 0."""
    e = np.zeros_like(r)
    s = r.copy()
    for _ in range(steps):
        q = A @ s
        qq = np.vdot(q, q).real
        if qq <= 0.0:
            break
        alpha = np.vdot(q, s) / qq
        e = e + alpha * s
        s = s - alpha * q
    return e


def sap_apply(U, dims, m0, v, block, cycles, mr_steps, antiperiodic=True):
    """M_SAP v for D_W(m0) (see the module docstring); v, result: [V, 4, 3] complex."""
    D = dense.wilson_matrix(U, dims, m0, antiperiodic)
    vv = np.asarray(v, dtype=np.complex128).reshape(-1)
    x = np.zeros_like(vv)
    parts = blocks(dims, block)
    sub = [(c, idx, D[idx][:, idx].tocsr()) for c, idx in parts]
    for _ in range(cycles):
        for colour in (0, 1):
            r = vv - D @ x
            for c, idx, Dbb in sub:
                if c == colour:
                    x[idx] += minimal_residual(Dbb, r[idx], mr_steps)
    return x.reshape(np.shape(v))

"""Free-field closed forms (U = I): the exact pins of the Wilson and overlap operators.

With all links equal to the identity, a plane wave psi(x) = exp(i p.x) u is
an eigenvector of D_W(m0) from Eq. (Wilson-Dirac) once u is an eigenvector
of sum_mu gamma_mu sin p_mu:

    D_W(m0) psi = (m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu) psi,

and (sum_mu gamma_mu s_mu)^2 = |s|^2 I by Eq. (commutativity_rel), so the
eigenvalue is lambda = m0 + sum_mu (1 - cos p_mu) +- i |s|. D_W is normal in
the free theory (Sec. 4), so by Theorem the:D_D_N_eigs the same psi is an
eigenvector of D_N with eigenvalue rho + csign(lambda), csign(z) = z/|z|.
Momenta: p_mu = 2 pi n_mu / L_mu, plus pi / L_0 in time when the time
boundary is antiperiodic.
"""

import itertools

import numpy as np

from .gamma import GAMMA


def momenta(dims, antiperiodic=True):
    out = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = np.array([(2 * np.pi * n[m] + (np.pi if (m == 0 and antiperiodic) else 0.0)) / dims[m]
                      for m in range(4)])
        out.append((n, p))
    return out


def wilson_eigs(dims, m0, antiperiodic=True):
    """All 12V free-field eigenvalues of D_W(m0) (each +-i|s| branch has multiplicity 6)."""
    ev = []
    for _, p in momenta(dims, antiperiodic):
        re = m0 + np.sum(1.0 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(p) ** 2))
        ev += [re + 1j * im] * 6 + [re - 1j * im] * 6
    return np.array(ev)


def overlap_eigs(dims, m0_ker, rho, antiperiodic=True):
    lam = wilson_eigs(dims, m0_ker, antiperiodic)
    return rho + lam / np.abs(lam)


def plane_wave_eigvec(dims, n, branch, colour, antiperiodic=True):
    """(psi [V][4][3], lambda_W without m0) for momentum index n.

    branch = +1/-1 selects the eigenvalue +-|s| of sum gamma_mu sin p_mu;
    the spin vector is the first such eigenvector from numpy's eigh.
    """
    dims = tuple(dims)
    p = np.array([(2 * np.pi * n[m] + (np.pi if (m == 0 and antiperiodic) else 0.0)) / dims[m]
                  for m in range(4)])
    G = sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    w, W = np.linalg.eigh(G)
    k = int(np.argmax(w)) if branch > 0 else int(np.argmin(w))
    u = np.zeros((4, 3), dtype=np.complex128)
    u[:, colour] = W[:, k]
    grids = np.meshgrid(*[np.arange(L) for L in dims], indexing="ij")
    phase = sum(p[m] * grids[m] for m in range(4))
    psi = np.exp(1j * phase).reshape(-1)[:, None, None] * u[None]
    lam0 = np.sum(1.0 - np.cos(p)) + 1j * w[k]
    return np.ascontiguousarray(psi), lam0

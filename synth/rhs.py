"""Seeded right-hand sides [n_rhs][V][4][3] complex128 (or [V][4][3])."""

import numpy as np


def rhs_gaussian(dims, seed, n_rhs=None):
    """Re and Im of every component i.i.d. N(0,1) (re drawn before im)."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    shape = (V, 4, 3) if n_rhs is None else (n_rhs, V, 4, 3)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return np.ascontiguousarray(re + 1j * im)


def rhs_point(dims, spin, colour, site=0):
    """delta_{x,site} delta_{s,spin} delta_{c,colour}."""
    V = int(np.prod(dims))
    b = np.zeros((V, 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def rhs_z2(dims, seed, n_rhs=None):
    """Real +-1 per component, seeded."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    shape = (V, 4, 3) if n_rhs is None else (n_rhs, V, 4, 3)
    return (1.0 - 2.0 * rng.integers(0, 2, size=shape)).astype(np.complex128)


def rhs_plane_wave(dims, n, u, antiperiodic_time=True):
    """psi(x) = exp(i p.x) u with p_mu = (2 pi n_mu + pi*[mu=0 and antiperiodic]) / L_mu.

    u is a (4, 3) complex spin-colour vector. Returns [V][4][3] and p.
    """
    dims = tuple(dims)
    p = np.array([(2.0 * np.pi * n[m] + (np.pi if (m == 0 and antiperiodic_time) else 0.0))
                  / dims[m] for m in range(4)])
    grids = np.meshgrid(*[np.arange(L) for L in dims], indexing="ij")
    phase = np.zeros(dims)
    for m in range(4):
        phase = phase + p[m] * grids[m]
    psi = np.exp(1j * phase).reshape(-1)[:, None, None] * np.asarray(u)[None, :, :]
    return np.ascontiguousarray(psi.astype(np.complex128)), p

"""Gauge observables of Sec. 4: plaquettes, Wilson action, non-normality.

Written independently of the input generator: the plaquette follows
Eq. (plaquette_def1), Q^{mu,nu}_x = U_nu(x) U_mu(x+nu) U_nu(x+mu)^H U_mu(x)^H.
"""

import numpy as np


def _shift(F, axis):
    """F(x + e_axis) on a periodic (L0,L1,L2,L3,...) array."""
    return np.roll(F, -1, axis=axis)


def _dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def plaquettes(U, dims):
    """Dict {(mu, nu): [L0,L1,L2,L3,3,3]} of first-quadrant plaquettes, mu < nu."""
    Uf = U.reshape(tuple(dims) + (4, 3, 3))
    out = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Umu, Unu = Uf[..., mu, :, :], Uf[..., nu, :, :]
            out[(mu, nu)] = Unu @ _shift(Umu, nu) @ _dag(_shift(Unu, mu)) @ _dag(Umu)
    return out


def wilson_action(U, dims):
    """S_W = sum_x sum_{mu<nu} Re tr(I - Q^{mu,nu}_x)  (Sec. 4)."""
    s = 0.0
    for Q in plaquettes(U, dims).values():
        s += np.sum(3.0 - np.trace(Q, axis1=-2, axis2=-1).real)
    return float(s)


def average_plaquette(U, dims):
    """Q_avg of Eq. (avgplaquette): mean of Re tr Q over the 6V plaquettes."""
    V = int(np.prod(dims))
    tot = sum(np.sum(np.trace(Q, axis1=-2, axis2=-1).real) for Q in plaquettes(U, dims).values())
    return float(tot) / (6 * V)


def nonnormality_from_plaquettes(U, dims):
    """Right-hand side of Eq. (deviationfromnormality): 16 * S_W."""
    return 16.0 * wilson_action(U, dims)

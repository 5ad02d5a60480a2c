"""Euclidean gamma matrices in a chiral basis (Sec. 2, Eq. commutativity_rel).

The paper fixes only the Clifford relations {gamma_mu, gamma_nu} = 2 delta_{mu nu}
and gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 (Eq. gamma_commutativity); the
basis is a free choice. This one is Hermitian with gamma_0 the time direction:

    gamma_0 = [[0, I], [I, 0]],  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]

which makes gamma_5 = diag(-1, -1, +1, +1).
"""

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]

GAMMA = [np.block([[_Z2, _I2], [_I2, _Z2]])] + [
    np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _SIGMA
]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=np.complex128)


def proj(mu, sign):
    """pi^{+-}_mu = (I + sign*gamma_mu)/2 (Appendix A)."""
    return 0.5 * (I4 + sign * GAMMA[mu])

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws gauge fields and right-hand sides. It holds none of the
overlap method's arithmetic (no Wilson-Dirac operator, no sign function, no
solver); it only produces the inputs both sides are run on.

Conventions (lattice of Sec. 2, x = (x0, x1, x2, x3) with x0 = time):
  * dims = (L0, L1, L2, L3); lexicographic site index
    s = ((x0*L1 + x1)*L2 + x2)*L3 + x3 (x3 fastest).
  * gauge field: complex128 array [V][4][3][3], U[s, mu, a, b] = row a,
    column b of the link U_mu(x) from x to x + mu-hat.
  * spinor field: complex128 array [V][4][3] (spin, colour), or
    [n_rhs][V][4][3] for several right-hand sides.
"""

from .gauge import (random_su3, gauge_field, stout_step, stout_smear,
                    random_gauge_rotation, gauge_transform_links,
                    gauge_transform_spinor)
from .rhs import rhs_gaussian, rhs_point, rhs_z2, rhs_plane_wave

__all__ = [
    "random_su3", "gauge_field", "stout_step", "stout_smear",
    "random_gauge_rotation", "gauge_transform_links", "gauge_transform_spinor",
    "rhs_gaussian", "rhs_point", "rhs_z2", "rhs_plane_wave",
]

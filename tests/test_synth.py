"""Input generator checks: SU(3) links, stout smearing lowers the Wilson action
(Sec. 4, Eq. stout and the Lie-Euler theorem), gauge rotations leave it fixed."""
import numpy as np

import synth
from oracle import observables

DIMS = (4, 4, 4, 4)


def _su3_err(U):
    Uh = np.conj(np.swapaxes(U, -1, -2))
    unit = np.abs(U @ Uh - np.eye(3)).max()
    det = np.abs(np.linalg.det(U) - 1.0).max()
    return unit, det


def test_random_links_are_su3_and_seeded():
    U = synth.gauge_field(DIMS, 0.3, 7)
    unit, det = _su3_err(U)
    assert unit < 1e-13 and det < 1e-13
    assert np.array_equal(U, synth.gauge_field(DIMS, 0.3, 7))
    assert not np.array_equal(U, synth.gauge_field(DIMS, 0.3, 8))


def test_stout_lowers_action_every_step_and_stays_su3():
    U = synth.gauge_field(DIMS, 0.5, 11)
    s = [observables.wilson_action(U, DIMS)]
    for _ in range(3):
        U = synth.stout_step(U, DIMS, 0.1)
        s.append(observables.wilson_action(U, DIMS))
    assert all(b < a for a, b in zip(s, s[1:])), s
    unit, det = _su3_err(U)
    assert unit < 1e-12 and det < 1e-12


def test_action_gauge_invariant():
    U = synth.gauge_field(DIMS, 0.5, 12)
    G = synth.random_gauge_rotation(DIMS, 13)
    Ug = synth.gauge_transform_links(U, DIMS, G)
    assert abs(observables.wilson_action(Ug, DIMS) - observables.wilson_action(U, DIMS)) < 1e-9


def test_rhs_shapes():
    b = synth.rhs_gaussian(DIMS, 1, n_rhs=3)
    assert b.shape == (3, 256, 4, 3)
    z = synth.rhs_z2(DIMS, 1)
    assert set(np.unique(z.real)) == {-1.0, 1.0} and np.all(z.imag == 0)
    p = synth.rhs_point(DIMS, 2, 1, site=5)
    assert p[5, 2, 1] == 1 and np.count_nonzero(p) == 1

"""Pins of the oracle's two-level multigrid preconditioner against independent facts:
  * the aggregates partition the dofs and each holds one chirality (gamma5 = -1 or +1);
  * P has orthonormal columns and spans the smoothed test vectors on every aggregate;
  * gamma5-hermiticity of D_W (Eq. gamma_5_symmetry) carries over to the coarse operator:
    with G = P^H Gamma5 P, which must be diagonal with entries -1/+1 by chirality,
    G D_c G = D_c^H (a chirality mix-up breaks both);
  * D_c couples a block only to itself and its nearest-neighbour blocks;
  * with an exact coarse solve the coarse correction is exact on range(P): the
    preconditioner maps D_W P y to P y;
  * with complete aggregates (n_v = aggregate size, P unitary) it is D_W^{-1};
  * m GMRES steps equal the least-squares minimiser over the explicit Krylov matrix
    [r, A'r, ..., A'^{m-1} r], A' = D_c M^{-1} (numpy lstsq, no Arnoldi);
  * as a stationary iteration it converges to D_W^{-1} b, in fewer iterations than the
    Schwarz smoother alone.
Three planted mistakes (a conjugate missing from the restriction, the wrong spin split for
the chiralities, the smoothing step applied with the wrong sign) each failed at least one
of these pins when this file was written.
"""
import numpy as np
import pytest

import synth
from oracle import amg, gamma


@pytest.fixture(scope="module")
def f4():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1301)
    start = synth.rhs_gaussian(dims, 1302, n_rhs=12)
    tl = amg.TwoLevel(U, dims, -0.3, start, 3, (2, 2, 2, 2), 2, 4, coarse_steps=None)
    return dims, U, tl


def test_aggregates_partition_by_chirality():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    aggs = amg.aggregates(dims, block)
    assert len(aggs) == 2 * 16
    allidx = np.sort(np.concatenate([idx for _, _, idx in aggs]))
    assert np.array_equal(allidx, np.arange(12 * 256))
    g5 = np.diag(gamma.GAMMA5).real
    for b, chi, idx in aggs:
        spins = (idx % 12) // 3
        assert set(np.unique(g5[spins])) == {-1.0 if chi == 0 else 1.0}


def test_prolongation_orthonormal_and_spans_test_vectors(f4):
    dims, U, tl = f4
    P = tl.P.toarray()
    assert np.allclose(P.conj().T @ P, np.eye(P.shape[1]), atol=1e-12)
    vecs = amg.smooth_test_vectors(U, dims, -0.3, synth.rhs_gaussian(dims, 1302, n_rhs=12), 3, (2, 2, 2, 2), 2, 4)
    # every smoothed vector lies in range(P): P P^H v = v
    assert np.linalg.norm(P @ (P.conj().T @ vecs) - vecs) < 1e-12 * np.linalg.norm(vecs)


def test_coarse_operator_is_gamma5_hermitian(f4):
    dims, U, tl = f4
    P = tl.P.toarray()
    G5 = np.kron(np.eye(256), np.kron(gamma.GAMMA5, np.eye(3)))
    G = P.conj().T @ G5 @ P
    nv = tl.nv
    expect = np.tile(np.concatenate([-np.ones(nv), np.ones(nv)]), 16)
    assert np.allclose(G, np.diag(expect), atol=1e-12)
    Dc = tl.Dc
    assert np.linalg.norm(G @ Dc @ G - Dc.conj().T) < 1e-12 * np.linalg.norm(Dc)


def test_coarse_operator_couples_nearest_neighbour_blocks():
    dims, block = (6, 4, 4, 4), (2, 2, 2, 2)          # 3 blocks in x0: blocks 0 and 2 differ
    U = synth.gauge_field(dims, 0.3, 1311)
    start = synth.rhs_gaussian(dims, 1312, n_rhs=3)
    tl = amg.TwoLevel(U, dims, -0.3, start, 1, block, 1, 2, coarse_steps=None)
    nb = [dims[m] // block[m] for m in range(4)]
    coords = [np.unravel_index(b, nb) for b in range(int(np.prod(nb)))]
    s = 2 * tl.nv
    for a, ca in enumerate(coords):
        for c, cc in enumerate(coords):
            d = [min((ca[m] - cc[m]) % nb[m], (cc[m] - ca[m]) % nb[m]) for m in range(4)]
            blk = tl.Dc[s * a:s * (a + 1), s * c:s * (c + 1)]
            if sum(d) > 1:
                assert np.abs(blk).max() == 0.0, (a, c)
            else:
                assert np.abs(blk).max() > 1e-3, (a, c)


def test_exact_coarse_correction_on_range_of_p(f4):
    dims, U, tl = f4
    rng = np.random.default_rng(5)
    y = rng.standard_normal(tl.P.shape[1]) + 1j * rng.standard_normal(tl.P.shape[1])
    Py = tl.P @ y
    out = tl.apply((tl.D @ Py).reshape(256, 4, 3)).reshape(-1)
    assert np.linalg.norm(out - Py) < 1e-11 * np.linalg.norm(Py)


def test_complete_aggregates_give_the_exact_inverse():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, 1321)
    nv = 16 * 6                                        # aggregate size: 16 sites x 2 spins x 3 colours
    start = synth.rhs_gaussian(dims, 1322, n_rhs=nv)
    tl = amg.TwoLevel(U, dims, -0.3, start, 0, block, 1, 2, coarse_steps=None)
    b = synth.rhs_gaussian(dims, 1323)
    x = tl.apply(b).reshape(-1)
    assert np.linalg.norm(tl.D @ x - b.reshape(-1)) < 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("m", [1, 3, 6])
def test_gmres_steps_equal_krylov_least_squares(f4, m):
    dims, U, tl = f4
    rng = np.random.default_rng(7)
    r = rng.standard_normal(tl.Dc.shape[0]) + 1j * rng.standard_normal(tl.Dc.shape[0])
    Ap = tl.Dc @ tl.Minv
    K = [r]
    for _ in range(m - 1):
        K.append(Ap @ K[-1])
    K = np.stack(K, axis=1)
    z = np.linalg.lstsq(Ap @ K, r, rcond=None)[0]
    ref = tl.Minv @ (K @ z)
    x = amg.gmres_steps(tl.Dc, r, tl.Minv, m)
    assert np.linalg.norm(x - ref) < 1e-9 * np.linalg.norm(ref)


def test_two_level_iteration_converges_faster_than_smoother(f4):
    dims, U, tl = f4
    b = synth.rhs_gaussian(dims, 1331).reshape(-1)
    xs = np.linalg.solve(tl.D.toarray(), b)

    def iterate(apply, n):
        x = np.zeros_like(b)
        for _ in range(n):
            x = x + apply((b - tl.D @ x).reshape(256, 4, 3)).reshape(-1)
        return np.linalg.norm(x - xs) / np.linalg.norm(xs)

    from oracle import sap
    e_mg = iterate(tl.apply, 8)
    e_sap = iterate(lambda r: sap.sap_apply(U, dims, -0.3, r, (2, 2, 2, 2), 2, 4), 8)
    assert e_mg < 1e-3 and e_mg < 0.1 * e_sap, (e_mg, e_sap)

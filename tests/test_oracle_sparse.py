"""Pins of the plain-C sparse oracle: agreement with the dense definition,
free-field closed form at volumes the dense oracle cannot reach, gauge
covariance, and the Zolotarev sign against the exact dense sign(Q)."""
import numpy as np
import pytest

import synth
from oracle import dense, freefield, sparse, zolotarev


def test_o2_gamma5_matches():
    assert np.allclose(sparse.gamma5_diag(), [-1, -1, 1, 1])


@pytest.mark.parametrize("dims,ap", [((4, 4, 4, 4), True), ((2, 4, 2, 6), False)])
def test_o2_wilson_equals_dense(dims, ap):
    U = synth.gauge_field(dims, 0.4, 41)
    psi = synth.rhs_gaussian(dims, 42)
    D = dense.wilson_matrix(U, dims, -0.8, antiperiodic=ap)
    ref = (D @ psi.reshape(-1)).reshape(psi.shape)
    out = sparse.wilson(psi, U, dims, -0.8, antiperiodic=ap)
    assert np.abs(out - ref).max() < 1e-14 * np.abs(ref).max() * 10


def test_o2_free_field_8x8x8x8():
    dims = (8, 8, 8, 8)
    V = 8 ** 4
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    for n, br, c in [((1, 0, 0, 0), 1, 0), ((5, 3, 2, 7), -1, 1)]:
        psi, lam0 = freefield.plane_wave_eigvec(dims, n, br, c)
        out = sparse.wilson(psi, U, dims, -1.0)
        assert np.abs(out - (lam0 - 1.0) * psi).max() < 1e-13


def test_o2_gauge_covariance_8x8x8x8():
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 51)
    G = synth.random_gauge_rotation(dims, 52)
    Ug = synth.gauge_transform_links(U, dims, G)
    psi = synth.rhs_gaussian(dims, 53)
    lhs = sparse.wilson(synth.gauge_transform_spinor(psi, G), Ug, dims, -1.0)
    rhs = synth.gauge_transform_spinor(sparse.wilson(psi, U, dims, -1.0), G)
    assert np.abs(lhs - rhs).max() < 1e-12


def test_o2_q2_hermitian_positive():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 61)
    a, b = synth.rhs_gaussian(dims, 62), synth.rhs_gaussian(dims, 63)
    qa, qb = sparse.q2_shift(a, U, dims, -1.0), sparse.q2_shift(b, U, dims, -1.0)
    assert abs(np.vdot(a, qb) - np.vdot(qa, b)) < 1e-11 * abs(np.vdot(a, qb))
    assert np.vdot(a, qa).real > 0


def test_o2_sign_matches_dense_sign():
    """Zolotarev + one CG per pole reproduces the exact W sign(Delta) W^H within
    the approximation error when [lam_min, lam_max] encloses spec |Q|."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    lmin, lmax = 0.98 * np.abs(w).min(), 1.02 * np.abs(w).max()
    co = zolotarev.zolotarev_coefficients(lmin / lmax, 20)
    b = synth.rhs_gaussian(dims, 2001)
    s, its = sparse.sign_zolo(b, U, dims, -1.0, lmin, co, 1e-13)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(s - ref) < 1e-11 * np.linalg.norm(ref)
    o, _ = sparse.overlap(b, U, dims, -1.0, rho, lmin, co, 1e-13)
    ref = (DN @ b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(o - ref) < 1e-11 * np.linalg.norm(ref)

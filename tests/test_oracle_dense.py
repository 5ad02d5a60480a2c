"""Pins of the dense FP64 oracle against what the paper and mathematics fix.

Each test names the passage it checks. A mistake in the oracle (a dropped
hopping term, a wrong sign, a transposed link, a wrong gamma matrix or
boundary phase) breaks at least one of them.
"""
import numpy as np
import pytest

import synth
from oracle import dense, freefield, observables
from oracle.gamma import GAMMA, GAMMA5, I4, proj

RHO_P = dense.rho_from_mu(0.05, -1.0)


def test_gamma_clifford_and_gamma5():
    """Eq. (commutativity_rel), Eq. (gamma_commutativity); gamma5 Hermitian, unitary."""
    for m in range(4):
        assert np.allclose(GAMMA[m], GAMMA[m].conj().T)
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2 * I4 * (m == n))
        assert np.allclose(GAMMA5 @ GAMMA[m], -GAMMA[m] @ GAMMA5)
    assert np.allclose(GAMMA5 @ GAMMA5, I4)
    assert np.allclose(GAMMA5, np.diag([-1, -1, 1, 1]))


def test_projectors_appendix_a():
    """Eq. (proj_relations): pi^+- are projections with pi^+ pi^- = 0, and the
    four identities of Appendix A for mu != nu."""
    for m in range(4):
        P, M = proj(m, +1), proj(m, -1)
        assert np.allclose(P @ P, P) and np.allclose(M @ M, M)
        assert np.allclose(P @ M, 0) and np.allclose(M @ P, 0)
        for n in range(4):
            if n == m:
                continue
            gm, gn = GAMMA[m], GAMMA[n]
            assert np.allclose(proj(m, -1) @ proj(n, -1) - proj(m, 1) @ proj(n, 1), 0.5 * (-gm - gn))
            assert np.allclose(proj(m, 1) @ proj(n, -1) - proj(m, -1) @ proj(n, 1), 0.5 * (gm - gn))


@pytest.fixture(scope="module")
def c1():
    """4^4, links exp(i 0.3 H), antiperiodic time, rho = 1, mu = 0.05."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    DN, S, w = dense.overlap_dense(U, dims, RHO_P, -1.0)
    return dims, U, DN, S, w


def test_matrix_size_4x4x4x4(c1):
    """Sec. 2: the 4^4 matrix has size 3072."""
    assert c1[2].shape == (3072, 3072)


def test_free_field_wilson_plane_waves():
    """Closed form of the free Wilson operator on plane waves (Eq. Wilson-Dirac with U = I)."""
    dims = (4, 4, 4, 8)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    D = dense.wilson_matrix(U, dims, -1.0)
    for n, br, c in [((0, 0, 0, 0), 1, 0), ((1, 2, 3, 5), -1, 2), ((3, 1, 0, 7), 1, 1)]:
        psi, lam0 = freefield.plane_wave_eigvec(dims, n, br, c)
        out = (D @ psi.reshape(-1)).reshape(psi.shape)
        assert np.allclose(out, (lam0 - 1.0) * psi, atol=1e-13)


def test_free_field_overlap_spectrum():
    """Theorem the:D_D_N_eigs in the free theory: spec(D_N) = rho + csign(spec D_W(m0))."""
    dims = (2, 2, 2, 4)
    V = int(np.prod(dims))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    DN, _, _ = dense.overlap_dense(U, dims, RHO_P, -1.0)
    ev = np.linalg.eigvals(DN)
    ref = freefield.overlap_eigs(dims, -1.0, RHO_P)
    key = lambda z: (np.round(z.real, 9), np.round(z.imag, 9))
    assert sorted(map(key, ev)) == sorted(map(key, ref))
    # the Wilson spectrum too
    evw = np.linalg.eigvals(dense.wilson_matrix(U, dims, -1.0).toarray())
    assert sorted(map(key, evw)) == sorted(map(key, freefield.wilson_eigs(dims, -1.0)))


def test_gamma5_hermiticity(c1):
    """Eq. (gamma_5_symmetry): (Gamma5 D_W)^H = Gamma5 D_W."""
    dims, U = c1[0], c1[1]
    Q = (dense.gamma5_matrix(256) @ dense.wilson_matrix(U, dims, -1.0)).toarray()
    assert np.abs(Q - Q.conj().T).max() < 1e-14


def test_sign_hermitian_involution(c1):
    """Sec. 2 / Lemma props_Wilson_Overlap(ii): sign(Q) Hermitian, sign(Q)^2 = I."""
    S = c1[3]
    assert np.abs(S - S.conj().T).max() < 1e-12
    assert np.abs(S @ S - np.eye(S.shape[0])).max() < 1e-11


def test_overlap_normal_and_on_circle(c1):
    """Lemma props_Wilson_Overlap(ii): D_N normal, eigenvalues on |lambda - rho| = 1,
    spectrum symmetric to the real axis."""
    DN = c1[2]
    assert np.abs(DN @ DN.conj().T - DN.conj().T @ DN).max() < 1e-11
    ev = np.linalg.eigvals(DN)
    assert np.abs(np.abs(ev - RHO_P) - 1.0).max() < 1e-10
    dist = np.abs(ev[:, None] - np.conj(ev)[None, :]).min(axis=1)
    assert dist.max() < 1e-8


def test_ginsparg_wilson(c1):
    """Eq. (GW) for D^ = D_N - (rho - 1) I (proof of Prop. neuberger), a = 1."""
    DN = c1[2]
    G5 = dense.gamma5_matrix(256).toarray()
    Dh = DN - (RHO_P - 1.0) * np.eye(DN.shape[0])
    assert np.abs(G5 @ Dh + Dh @ G5 - Dh @ G5 @ Dh).max() < 1e-11


def test_sign_equals_svd_polar_factor(c1):
    """Lemma svd_kernel / Prop. neuberger: Gamma5 sign(Q) = D_W (D_W^H D_W)^(-1/2)
    = U_svd V_svd^H, computed here with numpy's SVD instead of eigh."""
    dims, U, _, S, _ = c1
    Dw = dense.wilson_matrix(U, dims, -1.0).toarray()
    Us, _, Vh = np.linalg.svd(Dw)
    G5 = dense.gamma5_matrix(256).toarray()
    assert np.abs(G5 @ S - Us @ Vh).max() < 1e-11


def test_wilson_spectrum_symmetries():
    """Lemma props_Wilson_Overlap(i): spec(D_W(m0)) symmetric to the real axis
    and to Re z = m0 + 4."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, 5)
    m0 = -1.0
    ev = np.linalg.eigvals(dense.wilson_matrix(U, dims, m0).toarray())
    key = lambda z: (np.round(z.real, 8), np.round(z.imag, 8))
    assert sorted(map(key, ev)) == sorted(map(key, np.conj(ev)))
    assert sorted(map(key, ev)) == sorted(map(key, 2 * (m0 + 4) - ev))


def test_nonnormality_equals_wilson_action():
    """Prop. Fnorm: ||D_W^H D_W - D_W D_W^H||_F^2 = 16 sum_x sum_{mu<nu} Re tr(I - Q)."""
    for dims, eps, seed, st in [((4, 4, 4, 4), 0.3, 21, 0), ((4, 4, 4, 6), 0.5, 22, 2)]:
        U = synth.gauge_field(dims, eps, seed, stout_steps=st)
        D = dense.wilson_matrix(U, dims, -0.7)
        C = (D.conj().T @ D - D @ D.conj().T).tocoo()
        lhs = float(np.sum(np.abs(C.data) ** 2))
        rhs = observables.nonnormality_from_plaquettes(U, dims)
        assert abs(lhs - rhs) < 1e-9 * rhs
    # and it vanishes for a pure gauge field (Sec. 4)
    dims = (4, 4, 4, 4)
    V = 256
    Uid = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    Ug = synth.gauge_transform_links(Uid, dims, synth.random_gauge_rotation(dims, 3))
    D = dense.wilson_matrix(Ug, dims, -1.0)
    C = (D.conj().T @ D - D @ D.conj().T).tocoo()
    assert np.sum(np.abs(C.data) ** 2) < 1e-20


def test_gauge_covariance():
    """D[U^G] (G psi) = G D[U] psi for D_W and D_N (pure-gauge remark, Sec. 4)."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.4, 31)
    G = synth.random_gauge_rotation(dims, 32)
    Ug = synth.gauge_transform_links(U, dims, G)
    psi = synth.rhs_gaussian(dims, 33)
    D, Dg = dense.wilson_matrix(U, dims, -1.0), dense.wilson_matrix(Ug, dims, -1.0)
    lhs = (Dg @ synth.gauge_transform_spinor(psi, G).reshape(-1)).reshape(psi.shape)
    rhs = synth.gauge_transform_spinor((D @ psi.reshape(-1)).reshape(psi.shape), G)
    assert np.abs(lhs - rhs).max() < 1e-13
    DN, _, _ = dense.overlap_dense(U, dims, RHO_P, -1.0)
    DNg, _, _ = dense.overlap_dense(Ug, dims, RHO_P, -1.0)
    lhs = (DNg @ synth.gauge_transform_spinor(psi, G).reshape(-1)).reshape(psi.shape)
    rhs = synth.gauge_transform_spinor((DN @ psi.reshape(-1)).reshape(psi.shape), G)
    assert np.abs(lhs - rhs).max() < 1e-11


def test_dense_solve(c1):
    """Eq. (linsys): the LU solution satisfies D_N psi = eta."""
    DN = c1[2]
    eta = synth.rhs_gaussian((4, 4, 4, 4), 2001)
    psi = dense.overlap_solve_dense(DN, eta)
    r = eta.reshape(-1) - DN @ psi.reshape(-1)
    assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(eta)


def test_rho_parametrisation():
    """Sec. 5: rho = (-mu/2 + m0)/(mu/2 + m0) >= 1 for m0 < 0; Table 1 BMW values."""
    assert abs(dense.rho_from_mu(0.05, -1.0) - 1.025 / 0.975) < 1e-15
    r = dense.rho_from_mu(0.0135778, -1.3)
    assert abs(r - (1.3 + 0.0067889) / (1.3 - 0.0067889)) < 1e-15 and r > 1


def test_default_prec_mass_sends_circle_to_one_value():
    """Eq. (default_m) and Sec. 3: g(z) = (rho + csign(z + m0_ker))/(z + m0_prec) maps
    the circle C(-m0_ker, omega) to 1/omega."""
    rho, m0k, smin = RHO_P, -1.0, 0.3
    m0p = dense.default_prec_mass(rho, m0k, smin)
    omega = -m0k - smin
    z = -m0k + omega * np.exp(1j * np.linspace(0, 2 * np.pi, 17))
    g = (rho + (z + m0k) / np.abs(z + m0k)) / (z + m0p)
    assert np.allclose(g, 1.0 / omega)

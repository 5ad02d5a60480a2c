"""Pins of the oracle's restarted Krylov sign function (Sec. 5.2).

Each pin fixes a different part of the method against something outside it:
  * the quadrature rule against z^{-1/2} itself;
  * one cycle on the whole space against the exact f(A) c (eigendecomposition);
  * plain restarts against the closed form of restarted Arnoldi for matrix functions,
    f_k = ||c|| [V_1 .. V_k] f(H_hat) e_1 with H_hat block lower bidiagonal
    (Eiermann and Ernst, SIAM J. Numer. Anal. 44, 2006), evaluated with scipy's sqrtm:
    a wrong sign, a dropped beta or a wrong row in the error weights breaks it;
  * thick restarts against the dense sign, with the error bound checked to be a bound
    after every cycle (a wrong start column s breaks convergence);
  * the 4^4 gauge-field Q against the dense oracle's sign(Q).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import dense
from oracle.krylov_sign import krylov_sign, quadrature


def _hermitian(n, lam, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    W, _ = np.linalg.qr(X)
    return (W * lam) @ W.conj().T, W


def _rhs(n, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=n) + 1j * rng.normal(size=n)


def _spectrum(n, lo, hi, seed, small=()):
    rng = np.random.default_rng(seed)
    lam = np.concatenate([rng.uniform(lo, hi, n // 2), -rng.uniform(lo, hi, n - n // 2)])
    lam[:len(small)] = small
    return lam


@pytest.mark.parametrize("lo,hi", [(1e-3, 1.0), (0.2, 60.0), (1e-4, 1e4)])
def test_quadrature_is_inverse_square_root(lo, hi):
    t, w = quadrature(lo, hi)
    z = np.exp(np.linspace(np.log(lo), np.log(hi), 2001))
    r = (w[None, :] / (z[:, None] + t[None, :])).sum(axis=1)
    assert np.max(np.abs(r * np.sqrt(z) - 1.0)) < 5e-15


def test_one_cycle_on_the_whole_space_is_exact():
    n = 48
    lam = _spectrum(n, 0.2, 2.0, 3)
    Q, W = _hermitian(n, lam, 4)
    b = _rhs(n, 5)
    x, info = krylov_sign(lambda v: Q @ v, b, 0.9 * 0.2 ** 2, 4.1, 1e-13, m=n, keep=0)
    exact = (W * np.sign(lam)) @ (W.conj().T @ b)
    assert info["converged"] and info["cycles"] == 1
    assert np.linalg.norm(x - exact) <= 1e-13 * np.linalg.norm(b)


def test_plain_restarts_equal_block_bidiagonal_closed_form():
    n, m, k_max = 120, 10, 4
    Q, _ = _hermitian(n, _spectrum(n, 0.3, 2.0, 6), 7)
    b = _rhs(n, 8)
    _, info = krylov_sign(lambda v: Q @ v, b, 0.9 * 0.3 ** 2, 4.1, 0.0, m=m, keep=0,
                          max_cycles=k_max, history=True)
    data = info["cycle_data"]
    assert not info["converged"] and len(data) == k_max
    c = Q @ b
    for k in range(1, k_max + 1):
        Hh = np.zeros((k * m, k * m), dtype=np.complex128)
        for i, (_, H, beta, s, _) in enumerate(data[:k]):
            assert s == 0
            Hh[i * m:(i + 1) * m, i * m:(i + 1) * m] = H
            if i + 1 < k:
                Hh[(i + 1) * m, i * m + m - 1] = beta     # A v_m^{(i)} couples to the next cycle's v_1
        e1 = np.zeros(k * m, dtype=np.complex128)
        e1[0] = 1.0
        closed = np.linalg.norm(c) * np.hstack([d[0] for d in data[:k]]) @ np.linalg.solve(sla.sqrtm(Hh), e1)
        assert np.linalg.norm(data[k - 1][4] - closed) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("keep", [0, 4, 8])
def test_thick_restarts_reach_dense_sign_and_bound_holds(keep):
    n = 200
    lam = _spectrum(n, 0.3, 3.0, 1, small=(0.05, -0.07, 0.1, -0.12))
    Q, W = _hermitian(n, lam, 2)
    b = _rhs(n, 9)
    exact = (W * np.sign(lam)) @ (W.conj().T @ b)
    x, info = krylov_sign(lambda v: Q @ v, b, 0.9 * 0.05 ** 2, 9.1, 1e-12, m=20, keep=keep,
                          history=True)
    assert info["converged"]
    assert np.linalg.norm(x - exact) <= 1e-12 * np.linalg.norm(b)
    for bound, d in zip(info["bounds"], info["cycle_data"]):
        assert np.linalg.norm(d[4] - exact) <= bound * (1 + 1e-8) + 1e-14 * np.linalg.norm(b)
    if keep:
        assert all(d[3] == keep for d in info["cycle_data"][1:])


def test_thick_restart_needs_fewer_products_with_small_eigenvalues():
    n = 200
    lam = _spectrum(n, 0.3, 3.0, 1, small=(0.05, -0.07, 0.1, -0.12))
    Q, _ = _hermitian(n, lam, 2)
    b = _rhs(n, 9)
    runs = [krylov_sign(lambda v: Q @ v, b, 0.9 * 0.05 ** 2, 9.1, 1e-10, m=20, keep=k)[1] for k in (0, 6)]
    assert runs[1]["matvecs"] < 0.5 * runs[0]["matvecs"]


def test_gauge_field_4x4x4x4_matches_dense_sign():
    """Q = Gamma5 D_W(-1) on the 4^4 field exp(i 0.3 H), antiperiodic time."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    Q = (dense.gamma5_matrix(int(np.prod(dims))) @ dense.wilson_matrix(U, dims, -1.0)).toarray()
    S, w = dense.sign_hermitian(Q)
    b = _rhs(Q.shape[0], 2001)
    lo, hi = np.abs(w).min(), np.abs(w).max()
    x, info = krylov_sign(lambda v: Q @ v, b, 0.9 * lo ** 2, 1.1 * hi ** 2, 1e-11, m=30, keep=8)
    assert info["converged"] and info["cycles"] > 1
    assert np.linalg.norm(x - S @ b) <= 1e-11 * np.linalg.norm(b)


def test_zero_rhs():
    Q, _ = _hermitian(10, _spectrum(10, 0.5, 1.0, 1), 1)
    x, info = krylov_sign(lambda v: Q @ v, np.zeros(10), 0.2, 1.1, 1e-12)
    assert np.all(x == 0) and info["cycles"] == 0

"""Pins of the oracle's GMRES/FGMRES against numpy's dense solve."""
import numpy as np

import synth
from oracle import dense, solvers


def test_gmres_matches_lu():
    rng = np.random.default_rng(0)
    n = 300
    A = 3 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = solvers.fgmres(lambda v: A @ v, b, 1e-12, restart=15)
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
    M = np.linalg.inv(A + 0.2 * np.diag(rng.standard_normal(n)))
    x2, info2 = solvers.fgmres(lambda v: A @ v, b, 1e-12, restart=15, precond=lambda v: M @ v)
    assert info2["converged"] and info2["iters"] < info["iters"]
    assert np.linalg.norm(x2 - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x2)


def test_overlap_gmres_matches_lu():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.3, 71)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, _, _ = dense.overlap_dense(U, dims, rho, -1.0)
    eta = synth.rhs_gaussian(dims, 72)
    x, info = solvers.fgmres(lambda v: (DN @ v.reshape(-1)).reshape(v.shape), eta, 1e-10, restart=100)
    ref = dense.overlap_solve_dense(DN, eta)
    assert info["converged"] and np.linalg.norm(x - ref) < 1e-8 * np.linalg.norm(ref)


def test_power_iteration_free_field_sigma_max():
    """Sec. 5.1: sigma~_max from power iterations; free field D_W(0) has
    largest real part 8 - sum(1 - cos) at the largest momentum."""
    dims = (4, 4, 4, 4)
    V = 256
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    D = dense.wilson_matrix(U, dims, 0.0, antiperiodic=False)
    v0 = synth.rhs_gaussian(dims, 3).reshape(-1)
    est = solvers.power_iteration_max_real(lambda v: D @ v, v0, 200)
    assert abs(est - 8.0) < 0.05

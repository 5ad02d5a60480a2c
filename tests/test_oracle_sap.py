"""Pins of the oracle's Schwarz (SAP) application against independent definitions:
  * MR steps on one block converge to the exact block solve (scipy spsolve), and one
    MR step is the closed form alpha r with alpha = <A r, r> / <A r, A r>;
  * one cycle with exact block solves is one block Gauss-Seidel step over the colour
    partition, red first: x_R = D_RR^{-1} v_R, x_B = D_BB^{-1} (v_B - D_BR x_R) (a wrong
    colour order, a stale residual or a block that leaks across its faces breaks it);
  * as a stationary iteration the cycles converge to D_W^{-1} v, also with an odd number
    of blocks in a direction (blocks of one colour then touch across the boundary).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import dense, sap


@pytest.fixture(scope="module")
def f4():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1201)
    v = synth.rhs_gaussian(dims, 1202)
    return dims, U, v


def test_blocks_partition_and_colours():
    parts = sap.blocks((6, 4, 4, 4), (2, 2, 2, 2))
    assert len(parts) == 3 * 2 * 2 * 2
    allidx = np.sort(np.concatenate([idx for _, idx in parts]))
    assert np.array_equal(allidx, np.arange(12 * 6 * 4 * 4 * 4))
    cols = [c for c, _ in parts]
    assert cols[0] == 0 and cols[1] == 1 and sum(cols) == 12
    for bad in ((4, 4, 4, 4), (3, 2, 2, 2)):
        with pytest.raises(ValueError):
            sap.blocks((4, 4, 4, 4), bad)


def test_mr_converges_to_block_solve(f4):
    dims, U, v = f4
    D = dense.wilson_matrix(U, dims, 0.5)
    c, idx = sap.blocks(dims, (2, 2, 2, 2))[5]
    A = D[idx][:, idx].tocsr()
    r = v.reshape(-1)[idx]
    exact = spla.spsolve(A.tocsc(), r)
    e = sap.minimal_residual(A, r, 40)   # converged to rounding; more steps underflow
    assert np.linalg.norm(e - exact) <= 1e-10 * np.linalg.norm(exact)
    q = A @ r
    one = sap.minimal_residual(A, r, 1)
    assert np.allclose(one, (np.vdot(q, r) / np.vdot(q, q).real) * r, rtol=1e-14, atol=0)


def test_one_cycle_is_red_black_block_gauss_seidel(f4):
    dims, U, v = f4
    D = dense.wilson_matrix(U, dims, 0.5)
    parts = sap.blocks(dims, (2, 2, 2, 2))
    R = np.sort(np.concatenate([idx for c, idx in parts if c == 0]))
    B = np.sort(np.concatenate([idx for c, idx in parts if c == 1]))
    vv = v.reshape(-1)
    xR = spla.spsolve(D[R][:, R].tocsc(), vv[R])
    xB = spla.spsolve(D[B][:, B].tocsc(), vv[B] - D[B][:, R] @ xR)
    ref = np.zeros_like(vv)
    ref[R], ref[B] = xR, xB
    got = sap.sap_apply(U, dims, 0.5, v, (2, 2, 2, 2), 1, 40).reshape(-1)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 4)])
def test_cycles_converge_to_wilson_inverse(dims):
    U = synth.gauge_field(dims, 0.3, 1203)
    v = synth.rhs_gaussian(dims, 1204)
    D = dense.wilson_matrix(U, dims, 0.5)
    exact = spla.spsolve(D.tocsc(), v.reshape(-1))
    got = sap.sap_apply(U, dims, 0.5, v, (2, 2, 2, 2), 40, 40).reshape(-1)
    assert np.linalg.norm(got - exact) <= 1e-9 * np.linalg.norm(exact)
    # an inexact application (the preconditioner's setting) still reduces the residual
    x1 = sap.sap_apply(U, dims, 0.5, v, (2, 2, 2, 2), 2, 6).reshape(-1)
    assert np.linalg.norm(v.reshape(-1) - D @ x1) < 0.2 * np.linalg.norm(v)

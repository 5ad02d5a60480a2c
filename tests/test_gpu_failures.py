"""Failure statuses of the solvers, each produced on the host side or by an iteration cap:
no test here faults, traps or hangs the GPU. After every failure the same context must
still give correct results.

  OVL_ENOCONV     the multishift iteration cap (max_ms_iter) in sign_apply, and the outer
                  iteration cap (max_iter) in ovl_solve, both with a finite best iterate;
  OVL_EBREAKDOWN  a right-hand side whose squared norm overflows FP64 makes the first CG
                  scalar non-finite;
  OVL_ETIMEOUT    the wall-clock limit max_seconds of ovl_solve.
A preconditioner capped at one Wilson iteration per application (prec_max_iter = 1) still
converges, only more slowly.
"""
import numpy as np
import pytest

import synth
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1410_7170_gb300 as ovl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def c1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    return dims, U, DN, S, np.abs(w)


def _params(aw, **kw):
    return ovl.params_default(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), **kw)


@pytest.mark.parametrize("arith", [ovl.OVL_ARITH_FP64, ovl.OVL_ARITH_FF, ovl.OVL_ARITH_FP32])
def test_multishift_iteration_cap_returns_enoconv_with_finite_output(c1, arith):
    dims, U, DN, S, aw = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, _params(aw, max_ms_iter=3, check_every=1))
    b = synth.rhs_gaussian(dims, 2001)
    out = torch.full_like(dev(b), float("nan"))
    st = ovl.lib().sign_apply_arith(op.ctx, ovl._ptr(out, True), ovl._ptr(dev(b)), 1e-10, arith)
    assert st == ovl.OVL_ENOCONV
    assert "max_ms_iter" in ovl.lib().ovl_last_error(op.ctx).decode()
    o = out.cpu().numpy()
    assert np.isfinite(o).all()
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    err = np.linalg.norm(o - ref) / np.linalg.norm(ref)
    assert 1e-6 < err < 2.0   # a rough approximation after three iterations, not garbage
    op.close()


def test_outer_iteration_cap_returns_enoconv_with_best_iterate(c1):
    dims, U, DN, S, aw = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, _params(aw, max_iter=1, precond=ovl.OVL_PREC_NONE))
    b = synth.rhs_gaussian(dims, 2001)
    x = torch.zeros_like(dev(b))
    st, stats = op.ovl_solve(x, dev(b), 1, 1e-10, check=False)
    assert st == ovl.OVL_ENOCONV
    xh = x.cpu().numpy()
    assert np.isfinite(xh).all()
    r = b.reshape(-1) - DN @ xh.reshape(-1)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel < 1.0                                   # one GMRES step reduced the residual
    assert abs(rel - stats["true_rel_resid"]) < 1e-6   # and the reported residual is the true one
    assert stats["outer_iters"] == 1
    op.close()


def test_breakdown_on_overflowing_norm_and_context_survives(c1):
    dims, U, DN, S, aw = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, _params(aw))
    b = synth.rhs_gaussian(dims, 2001)
    huge = dev(b * 1e200)          # finite entries, ||b||^2 = inf in FP64
    out = torch.empty_like(huge)
    for arith in (ovl.OVL_ARITH_FP64, ovl.OVL_ARITH_FF):
        st = ovl.lib().sign_apply_arith(op.ctx, ovl._ptr(out, True), ovl._ptr(huge), 1e-10, arith)
        assert st == ovl.OVL_EBREAKDOWN, arith
        assert "breakdown" in ovl.lib().ovl_last_error(op.ctx).decode()
    # the context still computes correct results afterwards
    op.sign_apply(out, dev(b), 1e-12)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(out.cpu().numpy() - ref) < 1e-10 * np.linalg.norm(ref)
    op.close()


def test_wall_clock_limit_returns_etimeout_and_context_survives():
    dims = (16, 16, 16, 16)
    U = dev(synth.gauge_field(dims, 0.5, 1002, stout_steps=3, device="cuda"))
    b = dev(synth.rhs_gaussian(dims, 2002))
    p = ovl.params_default(precision=ovl.OVL_FP64, precond=ovl.OVL_PREC_NONE, max_seconds=1e-3)
    op = ovl.Overlap(U, dims, 1.0, 0.01, p)
    x = torch.zeros_like(b)
    st, _ = op.ovl_solve(x, b, 1, 1e-8, check=False)
    assert st == ovl.OVL_ETIMEOUT
    assert "max_seconds" in ovl.lib().ovl_last_error(op.ctx).decode()
    # the same context still applies the operator (the limit applies to ovl_solve only)
    s1 = torch.empty_like(b)
    s2 = torch.empty_like(b)
    op.sign_apply(s1, b, 1e-10)
    op.sign_apply(s2, s1, 1e-10)
    assert ((s2 - b).norm() / b.norm()).item() < 1e-8
    op.close()


def test_one_wilson_iteration_per_preconditioner_still_converges(c1):
    dims, U, DN, S, aw = c1
    b = synth.rhs_gaussian(dims, 2001)
    xs = dense.overlap_solve_dense(DN, b)
    its = {}
    for cap in (1, 64):
        p = _params(aw, precond=ovl.OVL_PREC_WILSON, precision=ovl.OVL_MIXED_FP32, prec_max_iter=cap)
        op = ovl.Overlap(U, dims, 1.0, 0.05, p)
        x = torch.zeros_like(dev(b))
        st, stats = op.ovl_solve(x, dev(b), 1, 1e-10)
        assert st == ovl.OVL_OK
        assert np.linalg.norm(x.cpu().numpy() - xs) < 1e-8 * np.linalg.norm(xs)
        its[cap] = stats["outer_iters"]
        op.close()
    assert its[1] >= its[64]

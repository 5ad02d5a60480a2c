"""GPU parity of the restarted Krylov sign function (Sec. 5.2) through the C ABI.

The library's OVL_SIGN_KRYLOV path against the oracle: the dense sign(Q) and D_N at 4^4
(exact up to the stopping bound), the oracle's own restarted Krylov sign with the same
cycle length, kept Ritz vectors and interval (same number of cycles, agreement to
rounding), and at 8^4 on a stout-smeared field the oracle's Krylov and Zolotarev signs.
Tolerance: 1e-10 relative (2-norm) per application at tol 1e-11, as for the Zolotarev
path; solves to 1e-8 relative solution error against dense LU.
"""
import numpy as np
import pytest

import synth
from oracle import dense, sparse, zolotarev
from oracle.krylov_sign import krylov_sign

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


def host(t):
    return t.cpu().numpy()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def c1():
    """4^4, links exp(i 0.3 H), antiperiodic time, rho = 1, mu = 0.05."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    Q = (dense.gamma5_matrix(int(np.prod(dims))) @ dense.wilson_matrix(U, dims, -1.0)).tocsr()
    return dims, U, DN, S, np.abs(w), Q


def kparams(aw, m, keep, **kw):
    return ovl.params_default(sign_method=ovl.OVL_SIGN_KRYLOV, krylov_m=m, krylov_keep=keep,
                              lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), **kw)


@pytest.mark.parametrize("m,keep", [(24, 0), (24, 8), (16, 14)])
def test_krylov_sign_matches_dense_and_oracle(c1, m, keep):
    dims, U, DN, S, aw, Q = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, kparams(aw, m, keep))
    b = synth.rhs_gaussian(dims, 2001)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-11)
    got = host(out).reshape(-1)
    cycles = op.krylov_sign_info()["cycles"]
    assert rel2(got, S @ b.reshape(-1)) < 1e-10
    ref, info = krylov_sign(lambda v: Q @ v, b.reshape(-1), (0.98 * aw.min()) ** 2, (1.02 * aw.max()) ** 2,
                            1e-11, m=m, keep=keep)
    print("4^4 m=%d keep=%d: cycles %d (oracle %d), |gpu - oracle| %.2e, |gpu - dense| %.2e"
          % (m, keep, cycles, info["cycles"], rel2(got, ref), rel2(got, S @ b.reshape(-1))))
    # both stop on the same error bound: the same cycle count up to a rounding tie
    assert info["converged"] and info["cycles"] > 1 and abs(cycles - info["cycles"]) <= 1
    assert rel2(got, ref) < 3e-11
    op.ovl_apply(out, dev(b), 1e-11)
    assert rel2(host(out).reshape(-1), DN @ b.reshape(-1)) < 1e-10
    op.close()


def test_krylov_sign_matches_oracles_8x8x8x8():
    """Stout-smeared 8^4 field: the oracle's Krylov sign with the same parameters and its
    Zolotarev sign (one plain CG per pole) agree with the GPU to the requested accuracy."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1102, stout_steps=3)
    lmin, lmax = 0.3, 7.0
    op = ovl.Overlap(U, dims, 1.0, 0.01, ovl.params_default(
        sign_method=ovl.OVL_SIGN_KRYLOV, krylov_m=40, krylov_keep=8, lambda_min=lmin, lambda_max=lmax))
    b = synth.rhs_gaussian(dims, 2102)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-10)
    got = host(out)
    V = int(np.prod(dims))
    g5 = sparse.gamma5_diag()

    def q_apply(v):
        return (sparse.wilson(v.reshape(V, 4, 3), U, dims, -1.0) * g5[None, :, None]).reshape(-1)

    ref, info = krylov_sign(q_apply, b.reshape(-1), lmin ** 2, lmax ** 2, 1e-10, m=40, keep=8)
    cycles = op.krylov_sign_info()["cycles"]
    co = zolotarev.zolotarev_coefficients(lmin / lmax, 16)
    zref, _ = sparse.sign_zolo(b, U, dims, -1.0, lmin, co, 1e-13)
    print("8^4: cycles %d (oracle %d), |gpu - oracle Krylov| %.2e, |gpu - oracle Zolotarev| %.2e"
          % (cycles, info["cycles"], rel2(got.reshape(-1), ref), rel2(got, zref)))
    assert info["converged"] and abs(cycles - info["cycles"]) <= 1
    assert rel2(got.reshape(-1), ref) < 3e-10
    assert rel2(got, zref) < 1e-9
    op.close()


@pytest.mark.parametrize("precond,precision", [(ovl.OVL_PREC_NONE, ovl.OVL_FP64),
                                               (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_FP32)])
def test_krylov_sign_solves_match_dense_lu(c1, precond, precision):
    """Outer D_N with the Krylov sign (two right-hand sides: the lock-step batch falls back to
    one at a time); in the recursive scheme the inner FP32 sign stays Zolotarev."""
    dims, U, DN, S, aw, Q = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, kparams(aw, 40, 8, precond=precond, precision=precision,
                                                 sap_block=(2, 2, 2, 2)))
    b = synth.rhs_gaussian(dims, 2005, n_rhs=2)
    x = torch.zeros_like(dev(b))
    st, stats = op.ovl_solve(x, dev(b), 2, 1e-11)
    for k in range(2):
        assert rel2(host(x[k]), dense.overlap_solve_dense(DN, b[k])) < 1e-8
    assert 0 < stats["ms_iters_fp64"] <= op.krylov_sign_info()["matvecs"]
    op.close()


def test_krylov_sign_with_deflation(c1):
    dims, U, DN, S, aw, Q = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, kparams(aw, 24, 8, n_deflate=8))
    b = synth.rhs_gaussian(dims, 2007)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-11)
    assert rel2(host(out).reshape(-1), S @ b.reshape(-1)) < 1e-10
    op.ovl_apply(out, dev(b), 1e-11)
    assert rel2(host(out).reshape(-1), DN @ b.reshape(-1)) < 1e-10
    op.close()


def test_krylov_sign_zero_rhs_and_parameter_checks(c1):
    dims, U, DN, S, aw, Q = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, kparams(aw, 24, 8))
    z = torch.zeros((int(np.prod(dims)), 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.ones_like(z)
    op.sign_apply(out, z, 1e-11)
    assert out.abs().max().item() == 0.0
    op.ovl_apply(out, z, 1e-11)
    assert out.abs().max().item() == 0.0
    assert op.krylov_sign_info()["cycles"] == 0
    op.close()
    for bad in ({"krylov_m": 121}, {"krylov_m": 3}, {"krylov_m": 24, "krylov_keep": 23},
                {"sign_method": 2}):
        kw = {"krylov_m": 24, "krylov_keep": 8}
        kw.update(bad)
        with pytest.raises(ovl.OvlError) as e:
            ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(sign_method=kw.pop("sign_method", 1), **kw))
        assert e.value.status == ovl.OVL_EINVAL

"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 path): 1e-13 relative (max-norm) for the Wilson stencil (only the
summation order differs), 1e-10 relative (2-norm) per sign / overlap application
(the stated per-apply bar; the Zolotarev error is below 1e-13 on the interval and the
multishift CG runs to 1e-12), 1e-8 relative solution error for solves.
"""
import numpy as np
import pytest

import synth
from oracle import dense, freefield, sparse, zolotarev

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


def params(**kw):
    kw.setdefault("lambda_min", 0.05)
    kw.setdefault("lambda_max", 8.0)
    return ovl.params_default(**kw)


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("tps", [1, 4])
@pytest.mark.parametrize("dims,ap,m0", [
    ((4, 4, 4, 4), True, -1.0),
    ((2, 6, 6, 10), True, 0.37),      # V = 720: ragged tail of the last block
    ((4, 2, 8, 6), False, -0.4),
    ((8, 8, 8, 8), True, -1.0),
    ((16, 16, 16, 16), True, -1.0),  # the 16^4 workload size
])
def test_wilson_apply_matches_oracle(dims, ap, m0, tps):
    U = synth.gauge_field(dims, 0.5, 100 + sum(dims), stout_steps=1)
    psi = synth.rhs_gaussian(dims, 200 + sum(dims))
    ref = sparse.wilson(psi, U, dims, m0, antiperiodic=ap)
    op = ovl.Overlap(U, dims, 1.0, 0.05, params(antiperiodic=int(ap), stencil_tps=tps))
    out = torch.empty_like(dev(psi))
    op.wilson_apply(out, dev(psi), m0)
    assert relmax(host(out), ref) < 1e-13
    # host (numpy) buffers through the same entry point
    out_h = np.empty_like(psi)
    op.wilson_apply(out_h, psi, m0)
    assert relmax(out_h, ref) < 1e-13
    op.close()


def test_wilson_free_field_32x32x32x32():
    """Closed form at the largest 4D workload size: plane waves are eigenvectors."""
    dims = (32, 32, 32, 32)
    V = 32 ** 4
    U = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    U[:, :, 0, 0] = 1
    U[:, :, 1, 1] = 1
    U[:, :, 2, 2] = 1
    op = ovl.Overlap(U, dims, 1.0, 0.02, params())
    for n, br, c in [((3, 1, 4, 1), 1, 0), ((31, 0, 17, 5), -1, 2)]:
        psi, lam0 = freefield.plane_wave_eigvec(dims, n, br, c)
        x = dev(psi)
        out = torch.empty_like(x)
        op.wilson_apply(out, x, -1.0)
        expect = (lam0 - 1.0) * x
        assert (out - expect).abs().max().item() < 1e-13
    op.close()


@pytest.fixture(scope="module")
def c1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    return dims, U, rho, DN, S, np.abs(w)


@pytest.mark.parametrize("tps", [1, 4])
def test_sign_apply_matches_dense_sign(c1, tps):
    dims, U, rho, DN, S, aw = c1
    p = params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), n_poles=20, stencil_tps=tps)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2001)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-12)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    assert rel2(host(out), ref) < 1e-10
    out2 = torch.empty_like(out)
    op.ovl_apply(out2, dev(b), 1e-12)
    ref2 = (DN @ b.reshape(-1)).reshape(b.shape)
    assert rel2(host(out2), ref2) < 1e-10
    op.close()


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8, 1e-10])
def test_adaptive_zolotarev_degree_keeps_accuracy(c1, tol):
    """With adaptive_poles each sign application uses the smallest degree whose uniform
    error is <= tol/10: the result still meets tol against the exact (dense) sign, and
    agrees with the fixed 20-pole result to about tol."""
    dims, U, rho, DN, S, aw = c1
    b = synth.rhs_gaussian(dims, 2005)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    outs = {}
    for adaptive in (0, 1):
        p = params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), n_poles=20, adaptive_poles=adaptive)
        op = ovl.Overlap(U, dims, 1.0, 0.05, p)
        out = torch.empty_like(dev(b))
        op.sign_apply(out, dev(b), tol)
        outs[adaptive] = host(out)
        assert rel2(outs[adaptive], ref) < 3 * tol, (adaptive, rel2(outs[adaptive], ref))
        op.close()
    assert rel2(outs[1], outs[0]) < 4 * tol


def test_lanczos_interval_encloses_spectrum(c1):
    dims, U, rho, DN, S, aw = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default())
    info = op.info()
    assert info["lambda_min"] <= aw.min() and info["lambda_max"] >= aw.max()
    assert info["lambda_min"] > 0.5 * aw.min() and info["lambda_max"] < 1.5 * aw.max()
    assert abs(info["rho"] - rho) < 1e-15
    # with the estimated interval the sign still meets the per-apply bar
    b = synth.rhs_gaussian(dims, 2002)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-12)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    assert rel2(host(out), ref) < 1e-10
    op.close()


def test_sigma_min_and_default_preconditioner_mass(c1):
    """m0_prec defaults to m0^def of Eq. (default_m) with sigma_min, the smallest real part of
    the eigenvalues of D_W(0), estimated by the smallest singular value of D_W(0). Both are
    checked against the dense oracle: the estimate matches the singular value (0.820 here), and
    lies within 0.2 of the exact smallest real part (0.692: the leftmost eigenvalues of this
    rough 4^4 field are a complex pair)."""
    dims, U, rho, DN, S, aw = c1
    DW0 = dense.wilson_matrix(U, dims, 0.0).toarray()
    smin_exact = np.linalg.svd(DW0, compute_uv=False).min()
    re_min = np.linalg.eigvals(DW0).real.min()
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(precond=ovl.OVL_PREC_WILSON))
    info = op.info()
    assert abs(info["sigma_min"] - smin_exact) < 1e-3 * smin_exact + 1e-4, (info["sigma_min"], smin_exact)
    assert abs(info["sigma_min"] - re_min) < 0.2, (info["sigma_min"], re_min)
    assert abs(info["m0_prec"] - dense.default_prec_mass(info["rho"], -1.0, info["sigma_min"])) < 1e-12
    op.close()
    # an explicit m0_prec wins; without a preconditioner no estimate is made
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(precond=ovl.OVL_PREC_WILSON, m0_prec=-0.3))
    assert op.info()["m0_prec"] == -0.3 and np.isnan(op.info()["sigma_min"])
    op.close()


def test_deflation_eigenpairs_match_dense(c1):
    """Low-mode deflation (Sec. 5.2): the k eigenvalues of Q = Gamma5 D_W(m0_ker) of smallest
    modulus match the dense oracle's, the eigenvectors have small residuals, and the sign
    interval then starts below |lambda_{k+1}|."""
    dims, U, rho, DN, S, aw = c1
    k = 16
    Q = dense.gamma5_matrix(int(np.prod(dims))) @ dense.wilson_matrix(U, dims, -1.0).toarray()
    lam = np.linalg.eigvalsh(0.5 * (Q + Q.conj().T))
    lam = lam[np.argsort(np.abs(lam))]
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(n_deflate=k))
    d = op.deflation_info()
    assert d["k"] == k and d["matvecs"] > 0 and d["setup_s"] > 0
    assert np.abs(np.array(d["lambda"]) - lam[:k]).max() < 1e-10
    assert abs(d["lambda_next"] - abs(lam[k])) < 1e-10
    assert d["resid_max"] < 1e-9
    info = op.info()
    assert info["lambda_min"] <= abs(lam[k]) and info["lambda_min"] >= 0.89 * abs(lam[k])
    op.close()


@pytest.mark.parametrize("precond,precision", [(ovl.OVL_PREC_NONE, ovl.OVL_FP64),
                                               (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_FP32)])
def test_deflated_sign_and_solve_match_dense(c1, precond, precision):
    """With 12 deflated eigenpairs the sign and D_N products still match the dense exact
    ones, and the solves match dense LU."""
    dims, U, rho, DN, S, aw = c1
    p = ovl.params_default(n_deflate=12, lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(),
                           precond=precond, precision=precision, sap_block=(2, 2, 2, 2))
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2007)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-12)
    assert rel2(host(out), (S @ b.reshape(-1)).reshape(b.shape)) < 1e-10
    op.ovl_apply(out, dev(b), 1e-12)
    assert rel2(host(out), (DN @ b.reshape(-1)).reshape(b.shape)) < 1e-10
    x = torch.zeros_like(dev(b))
    op.ovl_solve(x, dev(b), 1, 1e-11)
    assert rel2(host(x), dense.overlap_solve_dense(DN, b)) < 1e-8
    op.close()


def test_deflation_cuts_multishift_work_16x16x16x16():
    """At 16^4 deflating 24 eigenpairs raises the sign interval's lower end and cuts the
    multishift iterations of a recursive mixed solve (only by a few per cent on this field,
    whose low spectrum of |Q| is dense); the true residual still meets tol."""
    dims = (16, 16, 16, 16)
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1002, stout_steps=3)).cuda()
    b = torch.from_numpy(synth.rhs_gaussian(dims, 2002)).cuda()
    stats = {}
    for k in (0, 24):
        op = ovl.Overlap(U, dims, 1.0, 0.01, ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE,
                                                                precision=ovl.OVL_MIXED_FP32, n_deflate=k))
        x = torch.zeros_like(b)
        st, stats[k] = op.ovl_solve(x, b, 1, 1e-10)
        r = torch.empty_like(b)
        op.ovl_apply(r, x, 1e-13)
        assert ((b - r).norm() / b.norm()).item() < 2e-10, stats[k]
        if k:
            d = op.deflation_info()
            assert d["lambda_next"] > op.info()["lambda_min"] and d["resid_max"] < 1e-8
        op.close()
    # the FP64-accuracy sign runs in float-float in the mixed solver (ff_outer, the default)
    tight = {k: stats[k]["ms_iters_fp64"] + stats[k]["ms_iters_ff"] for k in stats}
    assert tight[24] < tight[0], stats
    assert stats[24]["ms_iters_low"] < stats[0]["ms_iters_low"], stats


def test_sign_apply_matches_sparse_oracle_8x8x8x8():
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1102, stout_steps=3)
    lmin, lmax = 0.3, 7.0
    p = params(lambda_min=lmin, lambda_max=lmax, n_poles=16)
    op = ovl.Overlap(U, dims, 1.0, 0.01, p)
    b = synth.rhs_gaussian(dims, 2102)
    out = torch.empty_like(dev(b))
    op.sign_apply(out, dev(b), 1e-12)
    co = zolotarev.zolotarev_coefficients(lmin / lmax, 16)
    ref, _ = sparse.sign_zolo(b, U, dims, -1.0, lmin, co, 1e-13)
    assert rel2(host(out), ref) < 1e-10
    op.close()


def test_sign_squares_to_identity_16x16x16x16():
    """Sec. 2: sign(Q)^2 = I, at the 16^4 workload size with the estimated interval."""
    dims = (16, 16, 16, 16)
    U = synth.gauge_field(dims, 0.5, 1002, stout_steps=3)
    op = ovl.Overlap(U, dims, 1.0, 0.01, ovl.params_default())
    b = dev(synth.rhs_gaussian(dims, 2003))
    s1 = torch.empty_like(b)
    s2 = torch.empty_like(b)
    op.sign_apply(s1, b, 1e-11)
    op.sign_apply(s2, s1, 1e-11)
    assert ((s2 - b).norm() / b.norm()).item() < 1e-9
    assert abs((s1.norm() / b.norm()).item() - 1.0) < 1e-9
    op.close()


def test_gmres_solve_matches_dense_lu(c1):
    """Config 1: 4^4, unpreconditioned GMRES(100) in FP64 against the dense LU solution."""
    dims, U, rho, DN, S, aw = c1
    p = params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), precond=ovl.OVL_PREC_NONE)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2001)
    x = torch.zeros_like(dev(b))
    st, stats = op.ovl_solve(x, dev(b), 1, 1e-11)
    ref = dense.overlap_solve_dense(DN, b)
    assert rel2(host(x), ref) < 1e-8
    r = b.reshape(-1) - DN @ host(x).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-10
    assert stats["outer_iters"] > 0 and stats["ms_iters_fp64"] > 0
    op.close()


@pytest.mark.parametrize("precond,precision,tps", [
    (ovl.OVL_PREC_WILSON, ovl.OVL_FP64, 1),
    (ovl.OVL_PREC_WILSON, ovl.OVL_MIXED_FP32, 4),
    (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_FP32, 1),
    (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_FP32, 4),
    (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_HALF, 1),
    (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_BF16, 1),
])
def test_preconditioned_solves_match_dense_lu(c1, precond, precision, tps):
    dims, U, rho, DN, S, aw = c1
    p = params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), precond=precond, precision=precision,
               sap_block=(2, 2, 2, 2), stencil_tps=tps)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2001)
    x = torch.zeros_like(dev(b))
    st, stats = op.ovl_solve(x, dev(b), 1, 1e-11)
    ref = dense.overlap_solve_dense(DN, b)
    assert rel2(host(x), ref) < 1e-8
    op.close()


def test_multiple_rhs_and_initial_guess(c1):
    dims, U, rho, DN, S, aw = c1
    p = params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max())
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2005, n_rhs=3)
    x = torch.zeros_like(dev(b))
    op.ovl_solve(x, dev(b), 3, 1e-11)
    for k in range(3):
        ref = dense.overlap_solve_dense(DN, b[k])
        assert rel2(host(x[k]), ref) < 1e-8
    # restarting from the solution converges at once
    st, stats = op.ovl_solve(x, dev(b), 3, 1e-9)
    assert stats["outer_iters"] == 0
    op.close()


def test_errors_are_reported_not_raised_on_device():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 5)
    bad = U.copy()
    bad[3, 1] *= 1.01
    with pytest.raises(ovl.OvlError) as e:
        ovl.Overlap(bad, dims, 1.0, 0.05, params())
    assert e.value.status == ovl.OVL_EINVAL
    with pytest.raises(ovl.OvlError):
        ovl.Overlap(U, (4, 4, 4, 3), 1.0, 0.05, params())
    op = ovl.Overlap(U, dims, 1.0, 0.05, params())
    b = synth.rhs_gaussian(dims, 6)
    b[7, 2, 1] = np.nan
    out = np.empty_like(b)
    with pytest.raises(ovl.OvlError) as e:
        op.wilson_apply(out, b, -1.0)
    assert e.value.status == ovl.OVL_EINVAL
    with pytest.raises(ovl.OvlError):
        op.sign_apply(out, synth.rhs_gaussian(dims, 7), 0.0)
    # the context is still usable after an argument error
    b2 = synth.rhs_gaussian(dims, 8)
    op.wilson_apply(out, b2, -1.0)
    assert relmax(out, sparse.wilson(b2, U, dims, -1.0)) < 1e-13
    op.close()


@pytest.mark.parametrize("precision,tol", [(ovl.OVL_MIXED_FP32, 1e-5), (ovl.OVL_FP64, 1e-10)])
def test_wilson_solve_residual_and_sap_quality(precision, tol):
    """The inexact Wilson solve (Sec. 5.1 preconditioner) reaches its tolerance, checked
    with the oracle's D_W; stronger Schwarz smoothing needs fewer outer iterations."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1202, stout_steps=3)
    b = synth.rhs_gaussian(dims, 2202)
    m0 = -0.3
    its = []
    for cyc, mr in [(1, 1), (2, 4)]:
        op = ovl.Overlap(U, dims, 1.0, 0.01, params(precision=precision, sap_cycles=cyc, sap_mr_iters=mr,
                                                    prec_max_iter=400, prec_restart=32))
        x = np.zeros_like(b)
        its.append(op.wilson_solve(x, b, m0, tol))
        r = b - sparse.wilson(x, U, dims, m0)
        assert np.linalg.norm(r) / np.linalg.norm(b) < tol * 1.5
        op.close()
    assert its[1] < its[0]


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (12, 8, 8, 8)])
def test_sap_threads_per_site_variants_agree(dims):
    """The FP32 Schwarz block kernel with 1, 2 or 4 threads per site computes the same
    smoother up to FP32 rounding (only the order of the hop sums differs). One FGMRES step
    (tol 0.9) returns a multiple of the smoother's output, so the solutions are compared
    directly; each variant then also solves to 1e-4 (checked with the oracle's D_W) in about the
    same number of iterations. With
    12 x 8^3 the blocks per direction are odd in x0, which takes the path that forms the
    residual on the whole lattice before the block solves."""
    U = synth.gauge_field(dims, 0.5, 1203, stout_steps=3)
    b = synth.rhs_gaussian(dims, 2203)
    m0 = -0.3
    one, its, res = {}, {}, {}
    for tps in (1, 2, 4):
        op = ovl.Overlap(U, dims, 1.0, 0.01, params(precision=ovl.OVL_MIXED_FP32, sap_tps=tps,
                                                    prec_max_iter=400, prec_restart=32))
        assert op.tuning_sap()["sap_tps"] == tps
        x = np.zeros_like(b)
        assert op.wilson_solve(x, b, m0, 0.9) in (1, 2)
        one[tps] = x
        x = np.zeros_like(b)
        its[tps] = op.wilson_solve(x, b, m0, 1e-4)
        r = b - sparse.wilson(x, U, dims, m0)
        res[tps] = np.linalg.norm(r) / np.linalg.norm(b)
        op.close()
    for tps in (2, 4):
        assert relmax(one[tps], one[1]) < 1e-5, (tps, relmax(one[tps], one[1]))
        assert abs(its[tps] - its[1]) <= 2, its
    assert max(res.values()) < 1.5e-4, res


@pytest.mark.parametrize("ff_outer", [0, 1])
def test_profiling_counters_are_consistent(ff_outer):
    """The instrumentation samples one multishift iteration per queued chunk: the timed
    launches are a subset of all launches, with positive times and bytes. The tight sign
    applications run in native FP64 (ff_outer = 0) or in float-float (ff_outer = 1)."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1204, stout_steps=3)
    b = torch.from_numpy(synth.rhs_gaussian(dims, 2204)).cuda()
    op = ovl.Overlap(torch.from_numpy(U).cuda(), dims, 1.0, 0.01,
                     ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE, precision=ovl.OVL_MIXED_FP32,
                                        ff_outer=ff_outer))
    op.prof_enable(True)
    op.prof_get(reset=True)
    x = torch.zeros_like(b)
    st, stats = op.ovl_solve(x, b, 1, 1e-8)
    pr = op.prof_get(reset=True)
    assert pr["valid"] == 1 and pr["launches"] > 0
    tight = "ff" if ff_outer else "f64"
    idle = "f64" if ff_outer else "ff"
    for name in ("ms_stencil_" + tight, "ms_shifts_" + tight, "ms_stencil_f32", "ms_shifts_f32"):
        k = pr[name]
        assert 0 < k["timed"] <= k["launches"], (name, k)
        assert k["ms"] > 0 and 0 < k["timed_bytes"] <= k["bytes"], (name, k)
    assert pr["ms_stencil_" + idle]["launches"] == 0 and pr["ms_shifts_" + idle]["launches"] == 0
    n_tight = stats["ms_iters_ff"] if ff_outer else stats["ms_iters_fp64"]
    assert pr["ms_stencil_" + tight]["launches"] == 2 * n_tight
    assert pr["ms_shifts_f32"]["launches"] == stats["ms_iters_low"]
    assert stats["t_sign_fp64"] > 0 and stats["t_sign_low"] > 0 and stats["t_prec"] > 0
    assert stats["t_sign_fp64"] + stats["t_sign_low"] + stats["t_prec"] <= stats["seconds"]
    op.close()


def test_autotuner_reports_a_choice():
    dims = (16, 16, 16, 16)
    U = synth.gauge_field(dims, 0.5, 7, stout_steps=0)
    op = ovl.Overlap(U, dims, 1.0, 0.01, params())
    t = op.tuning()
    assert t["tps64"] in (1, 4) and t["tps32"] in (1, 4)
    assert all(m > 0 for m in t["ms"])
    t = op.tuning_mrhs()   # multi-RHS kernels: the fastest of the three per right-hand side, at 4 and 12
    assert t["kernel"] in (1, 2, 3) and t["kernel_large"] in (1, 2, 3)
    assert all(m > 0 for m in t["ms4"] + t["ms12"])
    assert t["ms4"][t["kernel"] - 1] == min(t["ms4"]) and t["ms12"][t["kernel_large"] - 1] == min(t["ms12"])
    op.close()
    with pytest.raises(ovl.OvlError) as e:
        ovl.Overlap(U, dims, 1.0, 0.01, params(mrhs_kernel=4))
    assert e.value.status == ovl.OVL_EINVAL
    op = ovl.Overlap(U, dims, 1.0, 0.01, params(precond=ovl.OVL_PREC_RECURSIVE, precision=ovl.OVL_MIXED_FP32))
    t = op.tuning_sap()
    assert t["sap_tps"] in (1, 2, 4) and all(m > 0 for m in t["ms"])
    assert t["ms"][(1, 2, 4).index(t["sap_tps"])] == min(t["ms"])
    op.close()


def test_config4_half_storage_full_size():
    """32^3 x 64, 3-stout links, mu = 0.01, one Z2 source: FP16-stored inner multishift,
    FP64 outer FGMRES, tol 1e-10. The oracle cannot solve at this size; the check is the
    true residual through the FP64 D_N (itself pinned to the oracle at smaller volumes), and
    that D_N's stencil on the solution against the oracle's definitional stencil on the whole
    lattice."""
    dims = (64, 32, 32, 32)
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1004, stout_steps=3, device="cuda")).cuda()
    b = torch.from_numpy(synth.rhs_z2(dims, 2004)).cuda()
    op = ovl.Overlap(U, dims, 1.0, 0.01, ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE,
                                                            precision=ovl.OVL_MIXED_HALF))
    x = torch.zeros_like(b)
    st, stats = op.ovl_solve(x, b, 1, 1e-10)
    r = torch.empty_like(b)
    op.ovl_apply(r, x, 1e-13)
    res = ((b - r).norm() / b.norm()).item()
    assert res < 2e-10, (res, stats)
    assert stats["ms_iters_low"] > 0
    w = torch.empty_like(x)
    op.wilson_apply(w, x, -1.0)
    ref = sparse.wilson(x.cpu().numpy(), U.cpu().numpy(), dims, -1.0)
    err = np.abs(w.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-12, err
    op.close()


@pytest.mark.parametrize("precision", [ovl.OVL_MIXED_FP32, ovl.OVL_MIXED_HALF, ovl.OVL_MIXED_BF16])
def test_16bit_storage_solves_16x16x16x16(precision):
    """16^4, 3-stout links, mu = 0.01: the recursive solver with FP32, FP16-stored and
    BF16-stored inner multishift directions reaches tol 1e-10 in the true FP64 residual,
    and the 16-bit modes use their lower-precision sign."""
    dims = (16, 16, 16, 16)
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1002, stout_steps=3)).cuda()
    b = torch.from_numpy(synth.rhs_gaussian(dims, 2002)).cuda()
    op = ovl.Overlap(U, dims, 1.0, 0.01, ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE, precision=precision))
    x = torch.zeros_like(b)
    st, stats = op.ovl_solve(x, b, 1, 1e-10)
    r = torch.empty_like(b)
    op.ovl_apply(r, x, 1e-13)
    res = ((b - r).norm() / b.norm()).item()
    assert res < 2e-10, (res, stats)
    assert stats["ms_iters_low"] > 0
    op.close()


def test_gauge_generator_torch_path_matches_numpy():
    """The device path of the input generator reproduces the numpy path to rounding."""
    dims = (4, 4, 4, 6)
    a = synth.gauge_field(dims, 0.5, 77, stout_steps=2)
    b = synth.gauge_field(dims, 0.5, 77, stout_steps=2, device="cuda")
    assert np.abs(a - b).max() < 1e-12


def test_edge_cases_zero_rhs_and_smallest_lattice():
    """Degenerate inputs: b = 0 gives x = 0 (and sign(Q) 0 = 0, D_N 0 = 0) without
    iterating; n_rhs = 0 is an argument error; the smallest lattice 2^4 (16 sites, wrap-around
    neighbours in every direction) matches the dense oracle for D_W, sign(Q) and the solve."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1206)
    op = ovl.Overlap(U, dims, 1.0, 0.05, params())
    z = torch.zeros((256, 4, 3), dtype=torch.complex128, device="cuda")
    x = torch.ones_like(z)
    st, stats = op.ovl_solve(x, z, 1, 1e-10)
    assert torch.count_nonzero(x).item() == 0 and stats["outer_iters"] == 0
    out = torch.ones_like(z)
    op.sign_apply(out, z, 1e-10)
    assert torch.count_nonzero(out).item() == 0
    op.ovl_apply(out, z, 1e-10)
    assert torch.count_nonzero(out).item() == 0
    with pytest.raises(ovl.OvlError) as e:
        op.ovl_solve(x, z, 0, 1e-10)
    assert e.value.status == ovl.OVL_EINVAL
    op.close()
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.3, 1207)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    aw = np.abs(w)
    op = ovl.Overlap(U, dims, 1.0, 0.05, params(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max()))
    b = synth.rhs_gaussian(dims, 2207)
    out = np.empty_like(b)
    op.wilson_apply(out, b, -1.0)
    assert relmax(out, sparse.wilson(b, U, dims, -1.0)) < 1e-13
    o = torch.empty_like(dev(b))
    op.sign_apply(o, dev(b), 1e-12)
    assert rel2(host(o), (S @ b.reshape(-1)).reshape(b.shape)) < 1e-10
    x = torch.zeros_like(dev(b))
    op.ovl_solve(x, dev(b), 1, 1e-11)
    assert rel2(host(x), dense.overlap_solve_dense(DN, b)) < 1e-8
    op.close()

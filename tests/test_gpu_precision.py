"""GPU parity of every arithmetic the solver uses, through the C ABI entry points that take
the arithmetic as an argument (wilson_apply_arith, wilson_apply_n_arith, sign_apply_arith),
against the CPU oracle.

The paper computes the outer D_N products in double precision and its preconditioner in
single precision (Sec. 5.2, Sec. 5.3 with Table 3). The library runs the FP64-accuracy
products in float-float arithmetic (pairs of FP32) and the inner ones in FP32, optionally
with FP16- or BF16-stored shifted directions. Each of these kernels is compared element by
element with the oracle here, not only through whole solves (where an FP64 outer solver
would absorb a wrong inner result as extra iterations).

Tolerances:
  stencil, float-float: 1e-13 relative max-norm (the FP64 bar; float-float carries ~48 bits);
  stencil, FP32: 5e-7 relative max-norm (inputs rounded to 24 bits, ~50 terms per output);
  stencil, 16-bit links and spinors: 3e-3 (FP16, 11 bits) and 2e-2 (BF16, 8 bits) relative
  max-norm, the inputs' rounding (about 5e-4 and 4e-3 per element) summed over ~50 terms;
  sign, float-float: 1e-10 relative 2-norm at tol 1e-12 (the FP64 per-apply bar);
  sign, FP32 / FP16-stored / BF16-stored: relative 2-norm error <= 3 x the requested
  accuracy, at every accuracy down to the floor the outer solver hands that arithmetic
  (1e-6, 1e-3, 1e-2).
"""
import numpy as np
import pytest

import synth
from oracle import dense, sparse, zolotarev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1410_7170_gb300 as ovl  # noqa: E402

FLOOR = {ovl.OVL_ARITH_FP32: 1e-6, ovl.OVL_ARITH_FP16: 1e-3, ovl.OVL_ARITH_BF16: 1e-2}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("arith,tps,bar", [
    (ovl.OVL_ARITH_FF, 1, 1e-13),
    (ovl.OVL_ARITH_FP32, 1, 5e-7),
    (ovl.OVL_ARITH_FP32, 4, 5e-7),
    (ovl.OVL_ARITH_FP16, 1, 3e-3),
    (ovl.OVL_ARITH_BF16, 1, 2e-2),
])
@pytest.mark.parametrize("dims,ap,m0", [
    ((4, 4, 4, 4), True, -1.0),
    ((2, 6, 6, 10), True, 0.37),     # V = 720: ragged tail of the last block
    ((4, 2, 8, 6), False, -0.4),
    ((8, 8, 8, 8), True, -1.0),
    ((16, 16, 16, 16), True, -1.0),
])
def test_wilson_arith_matches_oracle(dims, ap, m0, arith, tps, bar):
    U = synth.gauge_field(dims, 0.5, 100 + sum(dims), stout_steps=1)
    psi = synth.rhs_gaussian(dims, 200 + sum(dims))
    ref = sparse.wilson(psi, U, dims, m0, antiperiodic=ap)
    p = ovl.params_default(lambda_min=0.05, lambda_max=8.0, antiperiodic=int(ap), stencil_tps=tps)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    out = torch.empty_like(dev(psi))
    op.wilson_apply_arith(out, dev(psi), m0, arith)
    assert relmax(host(out), ref) < bar, relmax(host(out), ref)
    op.close()


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 7, 12, 13])
def test_wilson_multi_rhs_fp32_matches_oracle(nrhs, kernel):
    """The three FP32 multi-RHS stencil kernels (right-hand-side pairs sharing each link load;
    32-site tiles with a warp per right-hand side; links staged in shared memory), blocks of up
    to 12 per launch (13 = a full block and a ragged one), every right-hand side against the
    oracle."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1300, stout_steps=1)
    psi = np.stack([synth.rhs_gaussian(dims, 1400 + k) for k in range(nrhs)])
    p = ovl.params_default(lambda_min=0.05, lambda_max=8.0, mrhs_kernel=kernel)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    t = op.tuning_mrhs()
    assert t["kernel"] == kernel and t["kernel_large"] == kernel
    out = torch.empty_like(dev(psi))
    op.wilson_apply_n_arith(out, dev(psi), nrhs, -0.7, ovl.OVL_ARITH_FP32)
    o = host(out)
    for k in range(nrhs):
        ref = sparse.wilson(psi[k], U, dims, -0.7)
        assert relmax(o[k], ref) < 5e-7, (k, relmax(o[k], ref))
    op.close()


def test_wilson_multi_rhs_fp32_at_32x32x32x32():
    """Full 32^4 size with 12 right-hand sides in one launch (the 12-point-source workload's
    stencil, with the kernel the autotuner picks): three of the outputs compared element by
    element with the oracle's definitional stencil on the whole lattice."""
    dims = (32, 32, 32, 32)
    U = synth.gauge_field(dims, 0.5, 1003, stout_steps=3, device="cuda")
    nrhs = 12
    psi = np.stack([synth.rhs_gaussian(dims, 2300 + k) for k in range(nrhs)])
    p = ovl.params_default(lambda_min=0.05, lambda_max=8.0)
    op = ovl.Overlap(dev(U), dims, 1.0, 0.02, p)
    out = torch.empty_like(dev(psi))
    op.wilson_apply_n_arith(out, dev(psi), nrhs, -1.0, ovl.OVL_ARITH_FP32)
    o = host(out)
    for k in (0, 5, 11):
        ref = sparse.wilson(psi[k], U, dims, -1.0)
        assert relmax(o[k], ref) < 5e-7, (k, relmax(o[k], ref))
    op.close()


@pytest.fixture(scope="module")
def c1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    return dims, U, S, np.abs(w)


def test_sign_float_float_matches_dense_sign(c1):
    dims, U, S, aw = c1
    p = ovl.params_default(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), n_poles=20)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2001)
    out = torch.empty_like(dev(b))
    op.sign_apply_arith(out, dev(b), 1e-12, ovl.OVL_ARITH_FF)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    assert rel2(host(out), ref) < 1e-10, rel2(host(out), ref)
    op.close()


@pytest.mark.parametrize("arith", [ovl.OVL_ARITH_FP32, ovl.OVL_ARITH_FP16, ovl.OVL_ARITH_BF16])
def test_low_precision_sign_matches_dense_sign(c1, arith):
    """Each low-precision sign meets every requested accuracy down to its floor (the most
    accurate request the solver sends it) against the exact dense sign."""
    dims, U, S, aw = c1
    p = ovl.params_default(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), n_poles=20)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    b = synth.rhs_gaussian(dims, 2007)
    ref = (S @ b.reshape(-1)).reshape(b.shape)
    out = torch.empty_like(dev(b))
    tols = [t for t in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6) if t >= FLOOR[arith]]
    for tol in tols:
        op.sign_apply_arith(out, dev(b), tol, arith)
        err = rel2(host(out), ref)
        assert err <= 3 * tol, (arith, tol, err)
    op.close()


@pytest.mark.parametrize("arith,tol,bar", [
    (ovl.OVL_ARITH_FF, 1e-12, 1e-10),
    (ovl.OVL_ARITH_FP32, 1e-6, 3e-6),
    (ovl.OVL_ARITH_FP16, 1e-3, 3e-3),
    (ovl.OVL_ARITH_BF16, 1e-2, 3e-2),
])
def test_sign_arith_matches_sparse_oracle_8x8x8x8(arith, tol, bar):
    """Smeared 8^4 field (mu = 0.01): every arithmetic against the oracle's Zolotarev sign
    with one plain FP64 CG per pole."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1102, stout_steps=3)
    lmin, lmax = 0.3, 7.0
    p = ovl.params_default(lambda_min=lmin, lambda_max=lmax, n_poles=16)
    op = ovl.Overlap(U, dims, 1.0, 0.01, p)
    b = synth.rhs_gaussian(dims, 2102)
    out = torch.empty_like(dev(b))
    op.sign_apply_arith(out, dev(b), tol, arith)
    co = zolotarev.zolotarev_coefficients(lmin / lmax, 16)
    ref, _ = sparse.sign_zolo(b, U, dims, -1.0, lmin, co, 1e-13)
    err = rel2(host(out), ref)
    assert err < bar, (arith, err)
    op.close()


def test_arith_arguments_rejected():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(lambda_min=0.05, lambda_max=8.0))
    b = dev(synth.rhs_gaussian(dims, 1))
    out = torch.empty_like(b)
    with pytest.raises(ovl.OvlError) as e:
        op.wilson_apply_arith(out, b, -1.0, 9)
    assert e.value.status == ovl.OVL_EINVAL
    with pytest.raises(ovl.OvlError) as e:
        op.wilson_apply_n_arith(out, b, 1, -1.0, ovl.OVL_ARITH_FF)
    assert e.value.status == ovl.OVL_EINVAL
    with pytest.raises(ovl.OvlError) as e:
        op.sign_apply_arith(out, b, 1e-6, 7)
    assert e.value.status == ovl.OVL_EINVAL
    op.close()

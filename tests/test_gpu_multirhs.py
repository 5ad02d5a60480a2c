"""Several right-hand sides: the multi-RHS Wilson stencil, the lock-step batched
multishift sign and the batched solvers, against the oracle (and against the
single-right-hand-side path for the same systems)."""
import numpy as np
import pytest

import synth
from oracle import dense, sparse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1410_7170_gb300 as ovl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_multi_rhs_stencil_matches_oracle():
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 501, stout_steps=1)
    B = synth.rhs_gaussian(dims, 502, n_rhs=13)          # crosses the 12-per-launch boundary
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(lambda_min=0.1, lambda_max=8.0))
    out = torch.empty((13,) + B.shape[1:], dtype=torch.complex128, device="cuda")
    op.wilson_apply_n(out, torch.from_numpy(B).cuda(), 13, -0.7)
    o = out.cpu().numpy()
    for k in range(13):
        ref = sparse.wilson(B[k], U, dims, -0.7)
        assert np.abs(o[k] - ref).max() < 1e-13 * np.abs(ref).max()
    op.close()


@pytest.fixture(scope="module")
def c1():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    rho = dense.rho_from_mu(0.05, -1.0)
    DN, S, w = dense.overlap_dense(U, dims, rho, -1.0)
    return dims, U, DN, np.abs(w)


def test_batched_overlap_apply_matches_dense(c1):
    dims, U, DN, aw = c1
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max()))
    B = synth.rhs_gaussian(dims, 601, n_rhs=5)
    out = np.empty_like(B)
    op.ovl_apply_n(out, B, 5, 1e-12)
    for k in range(5):
        ref = (DN @ B[k].reshape(-1)).reshape(B[k].shape)
        assert rel2(out[k], ref) < 1e-10
    op.close()


@pytest.mark.parametrize("precond,precision", [
    (ovl.OVL_PREC_NONE, ovl.OVL_FP64),
    (ovl.OVL_PREC_WILSON, ovl.OVL_FP64),
    (ovl.OVL_PREC_RECURSIVE, ovl.OVL_MIXED_FP32),
])
def test_batched_solve_matches_dense_lu_and_single(c1, precond, precision):
    dims, U, DN, aw = c1
    kw = dict(lambda_min=0.98 * aw.min(), lambda_max=1.02 * aw.max(), precond=precond, precision=precision,
              sap_block=(2, 2, 2, 2))
    B = synth.rhs_gaussian(dims, 701, n_rhs=4)
    opb = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(rhs_block=12, **kw))
    xb = torch.zeros((4,) + B.shape[1:], dtype=torch.complex128, device="cuda")
    st, stats = opb.ovl_solve(xb, torch.from_numpy(B).cuda(), 4, 1e-10)
    ops = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(rhs_block=1, **kw))
    xs = torch.zeros_like(xb)
    ops.ovl_solve(xs, torch.from_numpy(B).cuda(), 4, 1e-10)
    for k in range(4):
        ref = dense.overlap_solve_dense(DN, B[k])
        assert rel2(xb[k].cpu().numpy(), ref) < 1e-8
        # the same system alone and in the batch: both within the tolerance of the solution
        assert rel2(xb[k].cpu().numpy(), xs[k].cpu().numpy()) < 2e-8
    opb.close()
    ops.close()


def test_config3_point_sources_batched_full_size():
    """32^4, 3-stout links, mu = 0.02, the 12 spin-colour point sources at the origin,
    batched (multi-RHS stencil, lock-step multishift), FP32 inner / FP64 outer, tol 1e-8.
    Checked through the FP64 D_N of the library on every right-hand side, and that D_N's stencil
    on two of the solutions against the oracle's definitional stencil on the whole lattice."""
    dims = (32, 32, 32, 32)
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1003, stout_steps=3, device="cuda")).cuda()
    B = torch.stack([torch.from_numpy(synth.rhs_point(dims, s, c)) for s in range(4) for c in range(3)]).cuda()
    op = ovl.Overlap(U, dims, 1.0, 0.02, ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE,
                                                            precision=ovl.OVL_MIXED_FP32, rhs_block=12))
    X = torch.zeros_like(B)
    st, stats = op.ovl_solve(X, B, 12, 1e-8)
    R = torch.empty_like(B)
    op.ovl_apply_n(R, X, 12, 1e-12)
    res = ((B - R).flatten(1).norm(dim=1) / B.flatten(1).norm(dim=1)).max().item()
    assert res < 2e-8, (res, stats)
    Uh = U.cpu().numpy()
    for k in (0, 7):
        w = torch.empty_like(X[k])
        op.wilson_apply(w, X[k], -1.0)
        ref = sparse.wilson(X[k].cpu().numpy(), Uh, dims, -1.0)
        err = np.abs(w.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 1e-12, (k, err)
    op.close()

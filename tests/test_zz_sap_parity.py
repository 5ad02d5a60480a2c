"""GPU parity of one Schwarz preconditioner application (the smoother of the Wilson
preconditioner, Sec. 5.1) through the C ABI against the oracle's red-black multiplicative
Schwarz with minimal-residual block solves.

Cases: an even number of blocks per direction (block residuals formed inside the block
kernel) and an odd one (one full-lattice residual per colour); FP64 and FP32 with 1, 2 and
4 threads per block site. Tolerances: FP64 1e-12 relative (2-norm; only the summation
order differs), FP32 5e-6 (the same algorithm run in complex64 on the host moves the result
by 1.6e-7).
"""
import numpy as np
import pytest

import synth
from oracle import sap

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


@pytest.mark.parametrize("dims,block,precision,cycles,mr,tps", [
    ((4, 4, 4, 4), (2, 2, 2, 2), ovl.OVL_FP64, 1, 4, 1),
    ((4, 4, 4, 4), (2, 2, 2, 2), ovl.OVL_FP64, 2, 6, 1),
    ((6, 4, 4, 4), (2, 2, 2, 2), ovl.OVL_FP64, 2, 6, 1),       # 3 blocks in x0
    ((8, 8, 8, 8), (4, 4, 4, 4), ovl.OVL_FP64, 2, 6, 1),
    ((8, 8, 8, 8), (4, 4, 4, 4), ovl.OVL_MIXED_FP32, 2, 6, 1),
    ((8, 8, 8, 8), (4, 4, 4, 4), ovl.OVL_MIXED_FP32, 2, 6, 2),
    ((8, 8, 8, 8), (4, 4, 4, 4), ovl.OVL_MIXED_FP32, 2, 6, 4),
    ((12, 8, 8, 8), (4, 4, 4, 4), ovl.OVL_MIXED_FP32, 2, 6, 1),  # 3 blocks in x0
])
def test_sap_application_matches_oracle(dims, block, precision, cycles, mr, tps):
    U = synth.gauge_field(dims, 0.5, 1300 + sum(dims), stout_steps=1)
    v = synth.rhs_gaussian(dims, 1400 + sum(dims))
    m0 = -0.3
    ref = sap.sap_apply(U, dims, m0, v, block, cycles, mr)
    p = ovl.params_default(precision=precision, sap_block=block, sap_cycles=cycles, sap_mr_iters=mr,
                           sap_tps=tps, lambda_min=0.05, lambda_max=8.0)
    op = ovl.Overlap(U, dims, 1.0, 0.05, p)
    out = torch.empty((int(np.prod(dims)), 4, 3), dtype=torch.complex128, device="cuda")
    op.sap_apply(out, torch.from_numpy(v).cuda(), m0)
    got = out.cpu().numpy()
    tol = 1e-12 if precision == ovl.OVL_FP64 else 5e-6
    err = rel2(got, ref)
    print("SAP %s %s %s cycles=%d mr=%d tps=%d: %.2e" % (dims, block, precision, cycles, mr, tps, err))
    assert err < tol
    # host buffers through the same entry point
    out_h = np.empty_like(v)
    op.sap_apply(out_h, v, m0)
    assert rel2(out_h, ref) < tol
    op.close()


def test_sap_application_rejects_bad_blocks():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1301)
    v = torch.from_numpy(synth.rhs_gaussian(dims, 1401)).cuda()
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(sap_block=(4, 4, 4, 4), sap_cycles=0,
                                                            lambda_min=0.05, lambda_max=8.0))
    with pytest.raises(ovl.OvlError) as e:
        op.sap_apply(torch.empty_like(v), v, -0.3)
    assert e.value.status == ovl.OVL_EINVAL
    op.close()

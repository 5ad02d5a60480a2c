"""wilson_apply_noalloc: the Wilson-Dirac operator for callers that cannot allocate
device memory (a runtime that owns all device memory through its own pool, or a
service loop where cudaFree's device-wide synchronisation is not allowed). Its output
must equal that of the context-based wilson_apply, call after call, although every
call reuses the same fixed working memory inside the library.

This file is collected last so that a run stopping at the first failure has already
run every other test."""
import numpy as np
import pytest

import synth
from oracle import sparse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1410_7170_gb300 as ovl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


@pytest.mark.parametrize("dims,ap,m0", [((8, 8, 8, 8), True, -1.0), ((2, 6, 6, 10), False, 0.37)])
def test_noalloc_matches_wilson_apply_on_consecutive_calls(dims, ap, m0):
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 300 + sum(dims), stout_steps=1)).cuda()
    ins = [torch.from_numpy(synth.rhs_gaussian(dims, 400 + k)).cuda() for k in range(2)]
    op = ovl.Overlap(U, dims, 1.0, 0.05, ovl.params_default(lambda_min=0.1, lambda_max=8.0,
                                                            antiperiodic=int(ap)))
    refs = []
    for x in ins:
        r = torch.empty_like(x)
        op.wilson_apply(r, x, m0)
        refs.append(r)
    op.close()
    outs = [torch.full_like(x, float("nan")) for x in ins]
    for x, o in zip(ins, outs):                 # two calls in a row on the same stream
        ovl.wilson_apply_noalloc(o, x, U, dims, m0, antiperiodic=ap)
    torch.cuda.synchronize()
    for x, o, r in zip(ins, outs, refs):
        assert torch.isfinite(o).all()
        err = ((o - r).abs().max() / r.abs().max()).item()
        assert err < 1e-13
        # and against the oracle's definitional stencil directly
        ref = sparse.wilson(x.cpu().numpy(), U.cpu().numpy(), dims, m0, antiperiodic=ap)
        oh = o.cpu().numpy()
        assert np.abs(oh - ref).max() < 1e-13 * np.abs(ref).max()


def test_noalloc_rejects_what_does_not_fit():
    dims = (16, 16, 16, 16)                      # 65536 sites > the fixed working memory
    V = 16 ** 4
    U = torch.zeros((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(ovl.OvlError) as e:
        ovl.wilson_apply_noalloc(x, x, U, dims, -1.0)
    assert e.value.status == ovl.OVL_EINVAL and "16384" in str(e.value)
    # buffers smaller than the lattice, or of another dtype, are refused before the call
    small = (4, 4, 4, 4)
    with pytest.raises(ValueError):
        ovl.wilson_apply_noalloc(x[:10], x[:256], U[:256], small, -1.0)
    with pytest.raises(ValueError):
        ovl.wilson_apply_noalloc(x[:256].to(torch.complex64), x[:256], U[:256], small, -1.0)
    small = (4, 4, 4, 4)
    Uh = synth.gauge_field(small, 0.3, 1)
    xh = synth.rhs_gaussian(small, 2)
    with pytest.raises(ovl.OvlError):            # host memory is not accepted
        ovl.wilson_apply_noalloc(np.empty_like(xh), xh, Uh, small, -1.0)

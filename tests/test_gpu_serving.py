"""Serving loop: requests of different lattices, masses and right-hand-side counts
arrive while others run; each result must equal (within the solve tolerance) the same
request solved alone; admission keeps the reserved memory within the HBM budget; faults
injected on the host (NaN right-hand side, non-SU(3) links, a request larger than the
budget) fail only their own request."""
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1410_7170_gb300 as ovl  # noqa: E402

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _requests(seed, n):
    rng = np.random.default_rng(seed)
    lattices = [(8, 8, 8, 8), (4, 4, 4, 8), (8, 8, 8, 4)]
    gauges = {d: synth.gauge_field(d, 0.5, 900 + i, stout_steps=3) for i, d in enumerate(lattices)}
    reqs = []
    for k in range(n):
        d = lattices[rng.integers(len(lattices))]
        mu = float(rng.choice([0.01, 0.05, 0.1]))
        nr = int(rng.integers(1, 4))
        b = synth.rhs_gaussian(d, 5000 + k, n_rhs=nr)
        reqs.append(dict(dims=d, gauge=gauges[d], key=1 + lattices.index(d), mu=mu, n_rhs=nr, b=b))
    return reqs


def _params():
    return ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE, precision=ovl.OVL_MIXED_FP32, rhs_block=4,
                              sap_block=(4, 4, 4, 4))


def test_mixed_stream_matches_each_request_alone():
    reqs = _requests(11, 10)
    p = _params()
    srv = ovl.Server(slots=3)
    rng = np.random.default_rng(12)
    tickets, outs = [], []
    for r in reqs:
        x = np.zeros_like(r["b"])
        outs.append(x)
        tickets.append(srv.submit(r["gauge"], r["dims"], 1.0, r["mu"], r["b"], x, r["n_rhs"], TOL, p,
                                  gauge_key=r["key"]))
        time.sleep(float(rng.exponential(0.02)))          # Poisson arrivals
    results = [srv.wait(t) for t in tickets]
    rep = srv.report()
    srv.close()
    assert rep["completed"] == len(reqs) and rep["failed"] == 0
    assert rep["p99_s"] >= rep["p50_s"] > 0 and rep["solves_per_s"] > 0
    print("serving report", rep)
    for r, x, res in zip(reqs, outs, results):
        assert res["status"] == ovl.OVL_OK, res["message"]
        op = ovl.Overlap(r["gauge"], r["dims"], 1.0, r["mu"], _params())
        xa = np.zeros_like(r["b"])
        op.ovl_solve(xa, r["b"], r["n_rhs"], TOL)
        for k in range(r["n_rhs"]):
            # the same kernels, launch shapes, batching and reduction orders run whatever else
            # is on the GPU, so the served result is the one computed alone, bit for bit
            d = np.linalg.norm(x[k] - xa[k]) / np.linalg.norm(xa[k])
            assert d == 0.0, (d, r["dims"], r["mu"], r["n_rhs"])
            # and the served result solves its system
            ax = np.empty_like(x[k])
            op.ovl_apply(ax, x[k], 1e-12)
            assert np.linalg.norm(r["b"][k] - ax) / np.linalg.norm(r["b"][k]) < 1.5 * TOL
        op.close()


def test_budget_admission_and_host_side_faults():
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 931, stout_steps=3)
    p = _params()
    good = [synth.rhs_gaussian(dims, 6000 + k, n_rhs=1) for k in range(3)]
    bad_b = synth.rhs_gaussian(dims, 6100, n_rhs=1)
    bad_b[0, 17, 2, 1] = np.nan
    bad_u = U.copy()
    bad_u[5, 2] *= 1.5
    # a budget that holds about one request at a time
    probe = ovl.Server(slots=1)
    x0 = np.zeros_like(good[0])
    t0 = probe.submit(U, dims, 1.0, 0.05, good[0], x0, 1, TOL, p)
    need = probe.wait(t0)["device_bytes"]
    probe.close()
    srv = ovl.Server(slots=3, hbm_budget=int(need * 1.5))
    xs = [np.zeros_like(b) for b in good]
    tk = [srv.submit(U, dims, 1.0, 0.05, b, x, 1, TOL, p) for b, x in zip(good, xs)]
    xb = np.zeros_like(bad_b)
    tb = srv.submit(U, dims, 1.0, 0.05, bad_b, xb, 1, TOL, p)
    xu = np.zeros_like(good[0])
    tu = srv.submit(bad_u, dims, 1.0, 0.05, good[0], xu, 1, TOL, p)
    with pytest.raises(ovl.OvlError) as e:          # can never fit the budget
        srv.submit(synth.gauge_field((16, 16, 16, 16), 0.5, 1), (16, 16, 16, 16), 1.0, 0.05,
                   synth.rhs_gaussian((16, 16, 16, 16), 1, n_rhs=1), np.zeros((1, 16 ** 4, 4, 3), np.complex128),
                   1, TOL, p)
    assert e.value.status == ovl.OVL_ENOMEM
    for t in tk:
        assert srv.wait(t)["status"] == ovl.OVL_OK
    rb, ru = srv.wait(tb), srv.wait(tu)
    assert rb["status"] == ovl.OVL_EINVAL and "NaN" in rb["message"]
    assert ru["status"] == ovl.OVL_EINVAL and "SU(3)" in ru["message"]
    rep = srv.report()
    assert rep["hbm_high_water"] <= int(need * 1.5)
    srv.close()
    for x in xs:
        assert np.all(np.isfinite(x)) and np.linalg.norm(x) > 0


def test_serving_full_size_range():
    """The serving configuration's size range: lattices 8^4 to 32^4 and 1 to 12 right-hand
    sides arrive together on 2 slots (the 32^4 gauge field is generated on the device). Every
    request completes, and every served solution meets the tolerance in the true FP64 residual
    of the library's own D_N."""
    specs = [((8, 8, 8, 8), 12, 0.05), ((24, 24, 24, 24), 2, 0.01), ((32, 32, 32, 32), 1, 0.02),
             ((16, 16, 16, 16), 4, 0.1), ((24, 24, 24, 24), 1, 0.05)]
    gauges = {}
    for i, (d, nr, mu) in enumerate(specs):
        if d not in gauges:
            dev = "cuda" if d[0] >= 24 else None
            gauges[d] = synth.gauge_field(d, 0.5, 950 + i, stout_steps=3, device=dev)
    p = _params()
    srv = ovl.Server(slots=2)
    tickets, outs, bs = [], [], []
    for k, (d, nr, mu) in enumerate(specs):
        b = torch.from_numpy(synth.rhs_gaussian(d, 6000 + k, n_rhs=nr)).cuda()
        x = torch.zeros_like(b)
        bs.append(b)
        outs.append(x)
        tickets.append(srv.submit(torch.from_numpy(gauges[d]).cuda(), d, 1.0, mu, b, x, nr, TOL, p,
                                  gauge_key=100 + list(gauges).index(d)))
    results = [srv.wait(t) for t in tickets]
    rep = srv.report()
    srv.close()
    assert rep["completed"] == len(specs) and rep["failed"] == 0, rep
    for (d, nr, mu), b, x, res in zip(specs, bs, outs, results):
        assert res["status"] == ovl.OVL_OK, res["message"]
        op = ovl.Overlap(torch.from_numpy(gauges[d]).cuda(), d, 1.0, mu, ovl.params_default())
        for k in range(nr):
            ax = torch.empty_like(x[k])
            op.ovl_apply(ax, x[k].contiguous(), 1e-12)
            rel = ((b[k] - ax).norm() / b[k].norm()).item()
            assert rel < 1.5 * TOL, (d, nr, mu, k, rel)
        op.close()

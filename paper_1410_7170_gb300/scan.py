"""Parameter scans of the overlap solver on one workload: the Wilson preconditioner mass
m0_prec (Sec. 5.1 scans [-sigma~_min, 0] and reports iterations and times) and the
relaxation factor of the sign accuracy (Sec. 5.2, Table 2 uses 1e-2).

    python -m paper_1410_7170_gb300.scan [--lattice 16x16x16x16] [--mu 0.01]
        [--m0 -0.6:0.0:0.05] [--relax 0.01,0.03,0.1,0.3] [--adapt] [--reps 3]
        [--set eps_inner=0.01,0.03 --set sap_mr_iters=4,6 --set sap_block=4x4x4x4,4x4x4x2 ...]

Each point is a full solve (outer FP64 FGMRES, recursive inner FP32 FGMRES, Wilson
preconditioner) of the seeded workload (links exp(i 0.5 H) smeared by 3 stout steps, one
Gaussian right-hand side, tol 1e-8), timed as the fastest of --reps solves after one
warm-up solve. One JSON line per point: the parameters, seconds per solve, outer, inner and
Wilson iterations, multishift iterations and the true residual. With --adapt a last line
gives the on-the-fly mass choice (params.m0_adapt) on the same workload. Each --set adds an
ovl_params field and its values to the grid (the inner FGMRES reduction eps_inner of Table 3,
the Wilson solve's eps_prec, prec_max_iter and Schwarz parameters of Sec. 5.1); the points are
the product of all lists.
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _range(spec):
    if ":" not in spec:
        return [float(v) for v in spec.split(",")]
    a, b, s = (float(v) for v in spec.split(":"))
    out, v = [], a
    while v <= b + 1e-12:
        out.append(round(v, 6))
        v += s
    return out


def main(argv=None):
    import torch

    import paper_1410_7170_gb300 as ovl
    import synth
    from paper_1410_7170_gb300 import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="16x16x16x16")
    ap.add_argument("--mu", type=float, default=0.01)
    ap.add_argument("--m0", default="", help="start:stop:step or a list of m0_prec (empty: m0^def only)")
    ap.add_argument("--relax", default="0.01", help="comma-separated relaxation factors")
    ap.add_argument("--adapt", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--set", action="append", default=[], help="field=v1,v2,... (repeatable)")
    a = ap.parse_args(argv)
    grid = [{}]
    for spec in a.set:
        key, vals = spec.split("=", 1)
        parsed = [tuple(int(u) for u in v.split("x")) if "x" in v else int(v) if v.lstrip("-").isdigit()
                  else float(v) for v in vals.split(",")]   # "4x4x4x2" for the array fields
        grid = [dict(g, **{key: v}) for g in grid for v in parsed]
    build.build()
    dims = tuple(int(v) for v in a.lattice.split("x"))
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1002, stout_steps=3, device="cuda")).cuda()
    b = torch.from_numpy(synth.rhs_gaussian(dims, 2002)).cuda()
    masses = _range(a.m0) if a.m0 else [float("nan")]
    relaxes = [float(v) for v in a.relax.split(",")]

    def run(**kw):
        p = ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE, precision=ovl.OVL_MIXED_FP32, **kw)
        op = ovl.Overlap(U, dims, 1.0, a.mu, p)
        best, stats = None, None
        for k in range(a.reps + 1):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, stats = op.ovl_solve(x, b, 1, 1e-8)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k > 0:
                best = dt if best is None else min(best, dt)
        info = op.info()
        extra = op.m0_adapt_info() if kw.get("m0_adapt") else None
        op.close()
        return best, stats, info, extra

    for r in relaxes:
        for m in masses:
            for extra in grid:
                kw = {"relax_factor": r, **extra}
                if m == m:   # not NaN
                    kw["m0_prec"] = m
                s, st, info, _ = run(**kw)
                print(json.dumps({"m0_prec": info["m0_prec"], "relax_factor": r, **extra, "s_per_solve": s,
                                  "outer": st["outer_iters"], "inner": st["inner_iters"], "wilson": st["prec_iters"],
                                  "ms_iters_tight": st["ms_iters_fp64"] + st["ms_iters_ff"],
                                  "ms_iters_low": st["ms_iters_low"], "true_rel_resid": st["true_rel_resid"]}),
                      flush=True)
    if a.adapt:
        s, st, info, extra = run(relax_factor=relaxes[0], m0_adapt=1)
        print(json.dumps({"m0_adapt": extra, "m0_def": info["m0_prec"], "relax_factor": relaxes[0],
                          "s_per_solve": s, "outer": st["outer_iters"], "inner": st["inner_iters"],
                          "wilson": st["prec_iters"], "true_rel_resid": st["true_rel_resid"]}), flush=True)


if __name__ == "__main__":
    main()

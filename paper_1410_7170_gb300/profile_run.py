"""Runs one operation of a workload through the library's public API, for external
profilers (ncu). Nothing is timed here; the benchmark is bench.py.

    python -m paper_1410_7170_gb300.profile_run --what solve_mixed|solve_fp64|sign64|sign_ff|sign64_krylov|sap|dslash64|dslash32|dslash_ff
        [--lattice 16x16x16x16] [--stout 3] [--stencil-tps 1] [--sap-tps 1] [--relax 0.3] [--m0-prec 0.0]

The gauge field, right-hand side and solver settings are those of bench.py's 16^4
workload (seeded links exp(i 0.5 H) smeared by 3 stout steps, rho = 1, mu = 0.01,
one Gaussian right-hand side, tol 1e-8, relaxation factor 0.3, and for the mixed solve the
Wilson preconditioner mass 0.0). Under a profiler the autotuner's timings are
distorted, so --stencil-tps / --sap-tps fix the kernel variants (0 = autotune).
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_1410_7170_gb300 as ovl
    import synth
    from paper_1410_7170_gb300 import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--what", required=True,
                    choices=["solve_mixed", "solve_fp64", "sign64", "sign_ff", "sign64_krylov", "sap", "dslash64",
                             "dslash32", "dslash_ff"])
    ap.add_argument("--lattice", default="16x16x16x16")
    ap.add_argument("--stout", type=int, default=3)
    ap.add_argument("--stencil-tps", type=int, default=0)
    ap.add_argument("--sap-tps", type=int, default=0)
    ap.add_argument("--relax", type=float, default=0.3)
    ap.add_argument("--m0-prec", type=float, default=0.0)
    a = ap.parse_args()
    build.build()
    dims = tuple(int(v) for v in a.lattice.split("x"))
    U = torch.from_numpy(synth.gauge_field(dims, 0.5, 1002, stout_steps=a.stout)).cuda()
    b = torch.from_numpy(synth.rhs_gaussian(dims, 2002)).cuda()
    tune = dict(stencil_tps=a.stencil_tps, sap_tps=a.sap_tps, relax_factor=a.relax)
    if a.what == "solve_mixed":
        p = ovl.params_default(precond=ovl.OVL_PREC_RECURSIVE, precision=ovl.OVL_MIXED_FP32, m0_prec=a.m0_prec, **tune)
    elif a.what == "solve_fp64":
        p = ovl.params_default(precond=ovl.OVL_PREC_WILSON, precision=ovl.OVL_FP64, prec_max_iter=4, **tune)
    elif a.what == "sign64_krylov":
        p = ovl.params_default(sign_method=ovl.OVL_SIGN_KRYLOV, **tune)
    elif a.what == "sap":
        p = ovl.params_default(precision=ovl.OVL_MIXED_FP32, **tune)
    else:
        p = ovl.params_default(**tune)
    op = ovl.Overlap(U, dims, 1.0, 0.01, p)
    x = torch.zeros_like(b)
    if a.what.startswith("solve"):
        st, stats = op.ovl_solve(x, b, 1, 1e-8)
        print(stats)
    elif a.what in ("sign64", "sign64_krylov"):
        op.sign_apply(x, b, 1e-8)
    elif a.what == "sign_ff":
        op.sign_apply_arith(x, b, 1e-8, ovl.OVL_ARITH_FF)
    elif a.what == "sap":
        op.sap_apply(x, b, -0.266)   # m0^def of the 16^4 workload field (Eq. default_m)
    else:
        print(op.dslash_time({"dslash64": 0, "dslash32": 1, "dslash_ff": 2}[a.what], 3), "ms")
    torch.cuda.synchronize()
    op.close()


if __name__ == "__main__":
    main()

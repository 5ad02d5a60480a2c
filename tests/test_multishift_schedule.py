"""The lagged schedule of the shifted-direction updates (the fused FP32 multishift iteration)
computes exactly what the three-kernel schedule computes.

Both schedules run the shifted CG recurrences with rescaled directions p~_l = p_l / zeta_l on a
small Hermitian positive matrix A (standing in for Q^2), in numpy FP64, the way the library's
kernels order them:

  three-kernel: alpha_k; r_{k+1}; beta_k and zeta_{k+1} (after the residual);
                y += w_l alpha_k zeta_{k+1} p~_l(k), p~_l(k+1) = r_{k+1} + b^l_k p~_l(k)
  lagged:       alpha_k and zeta_{k+1} (after the stencil); then, in the residual step,
                p~_l(k) = r_k + b^l_{k-1} p~_l(k-1), y += w_l alpha_k zeta_{k+1} p~_l(k),
                r_{k+1}; beta_k and b^l_k

Every update uses the same operands in the same order, so y agrees bit for bit, with the
drop rule on or off; and y is the rational function b + sum_l w_l (A + sigma_l)^{-1} b to the
solver tolerance."""
import numpy as np
import pytest


def _problem(n=48, seed=3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    lam = np.geomspace(0.05, 8.0, n) ** 2           # spectrum of Q^2 on the sign interval
    A = (Q * lam) @ Q.conj().T
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    sigma = np.array([0.0005, 0.004, 0.03, 0.3, 3.0, 30.0])
    w = np.array([0.2, 0.3, 0.5, 0.9, 1.5, 3.0])
    crit = np.full(len(sigma), 1.0)
    return A, b, sigma, w, crit


def _zeta_next(z, zp, a, ap, bp, ds):
    den = a * bp * (zp - z) + zp * ap * (1.0 + ds * a)
    return z * zp * ap / den if den != 0.0 else 0.0


def _three_kernel(A, b, sigma, w, crit, tol, iters, drop):
    n = len(sigma)
    r = b.copy(); y = b.copy(); P = [b.copy() for _ in range(n)]
    rr = pp = bb = np.vdot(b, b).real
    z = np.ones(n); zp = np.ones(n); ap, bp = 1.0, 0.0
    active = [True] * n
    for _ in range(iters):
        t = A @ P[0]
        a = rr / (np.vdot(P[0], t).real + sigma[0] * pp)
        r = r - a * (t + sigma[0] * P[0])
        rr_new = np.vdot(r, r).real
        beta = rr_new / rr
        upd = []
        for l in range(n):
            if not active[l]:
                continue
            zn = 1.0 if l == 0 else _zeta_next(z[l], zp[l], a, ap, bp, sigma[l] - sigma[0])
            ratio = zn / z[l] if z[l] != 0.0 else 0.0
            upd.append((l, a * zn, beta * ratio))
            zp[l], z[l] = z[l], zn
        for l, al, bl in upd:
            y = y + (w[l] * al) * P[l]
            P[l] = r + bl * P[l]
        if drop:
            live = [l for l, _, _ in upd if crit[l] * abs(z[l]) * np.sqrt(rr_new) > tol * np.sqrt(bb)]
            for l, _, _ in upd:
                if l > 0 and l not in live:
                    active[l] = False
            if not live:
                break
        ap, bp, pp, rr = a, beta, rr_new + beta * beta * pp, rr_new
    return y


def _lagged(A, b, sigma, w, crit, tol, iters, drop):
    n = len(sigma)
    r = b.copy(); y = b.copy(); P = [b.copy() for _ in range(n)]
    rr = pp = bb = np.vdot(b, b).real
    z = np.ones(n); zp = np.ones(n); ap, bp = 1.0, 0.0
    bl_prev = np.zeros(n)                            # b^l_{k-1}; zero before the first iteration
    active = [True] * n
    for _ in range(iters):
        t = A @ P[0]
        a = rr / (np.vdot(P[0], t).real + sigma[0] * pp)
        al = {}
        for l in range(n):                           # end of the stencil kernel: zeta_{k+1}
            if not active[l]:
                continue
            zn = 1.0 if l == 0 else _zeta_next(z[l], zp[l], a, ap, bp, sigma[l] - sigma[0])
            al[l] = a * zn
            zp[l], z[l] = z[l], zn
        for l in al:                                 # residual kernel: the lagged updates
            if l > 0:
                P[l] = r + bl_prev[l] * P[l]
            y = y + (w[l] * al[l]) * P[l]
        r_new = r - a * (t + sigma[0] * P[0])
        rr_new = np.vdot(r_new, r_new).real
        beta = rr_new / rr
        for l in al:
            bl_prev[l] = beta * (z[l] / zp[l] if zp[l] != 0.0 else 0.0)
        P[0] = r_new + bl_prev[0] * P[0]             # the p_0 update of the third kernel
        r = r_new
        if drop:
            live = [l for l in al if crit[l] * abs(z[l]) * np.sqrt(rr_new) > tol * np.sqrt(bb)]
            for l in al:
                if l > 0 and l not in live:
                    active[l] = False
            if not live:
                break
        ap, bp, pp, rr = a, beta, rr_new + beta * beta * pp, rr_new
    return y


@pytest.mark.parametrize("drop", [False, True])
def test_lagged_schedule_is_the_same_arithmetic(drop):
    A, b, sigma, w, crit = _problem()
    tol = 1e-10
    y3 = _three_kernel(A, b, sigma, w, crit, tol, 400, drop)
    yl = _lagged(A, b, sigma, w, crit, tol, 400, drop)
    assert np.array_equal(y3, yl)
    exact = b + sum(wl * np.linalg.solve(A + s * np.eye(len(b)), b) for s, wl in zip(sigma, w))
    assert np.linalg.norm(yl - exact) < 1e-8 * np.linalg.norm(exact)

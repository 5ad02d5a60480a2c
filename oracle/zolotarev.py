"""Zolotarev's optimal rational approximation of sign(x) (oracle copy).

Not part of the paper (Sec. 5.2 uses a thick-restart Krylov method for the
sign function); this is the approximation the GPU path evaluates. Zolotarev
(1877) gives the best uniform approximation of sign(x) on
[-1/k, -1] u [1, 1/k] of type (2n+1, 2n) in x as

    R(x) = d0 * x * prod_{l=1..n} (x^2 + c_{2l}) / prod_{l=1..n} (x^2 + c_{2l-1}),
    c_j  = sn^2(j K'/(2n+1); k') / cn^2(j K'/(2n+1); k'),  j = 1..2n,

with k' = sqrt(1 - k^2) and K' = K(k') the complete elliptic integral. The
scale d0 is the one that centres the error: here it is found by evaluating
x*prod(...) on a dense logarithmic grid of [1, 1/k] and taking
d0 = 2 / (max + min), so that 1 - R(x) equioscillates between +-delta.

Elliptic functions come from scipy.special (ellipk, ellipj), whose parameter
is m = k'^2. In partial fractions

    R(x) = d0 * x * (1 + sum_l a_l / (x^2 + c_{2l-1})),
    a_l  = prod_i (c_{2i} - c_{2l-1}) / prod_{i != l} (c_{2i-1} - c_{2l-1}).

For a Hermitian Q with spectrum of |Q| in [lam_min, lam_max], x = Q/lam_min:

    sign(Q) b ~= (d0/lam_min) Q [ b + sum_l a_l lam_min^2 (Q^2 + lam_min^2 c_{2l-1})^{-1} b ].
"""

import numpy as np
from scipy.special import ellipj, ellipk


def zolotarev_coefficients(k, n, grid=200001):
    """Coefficients for sign on [1, 1/k] (scaled by lam_min); 0 < k < 1."""
    if not (0.0 < k < 1.0) or n < 1:
        raise ValueError("need 0 < k < 1 and n >= 1")
    m = 1.0 - k * k
    Kp = ellipk(m)
    j = np.arange(1, 2 * n + 1)
    sn, cn, dn, _ = ellipj(j * Kp / (2 * n + 1), m)
    c = (sn / cn) ** 2
    c_den = c[0::2].copy()          # c_1, c_3, ..., c_{2n-1}
    c_num = c[1::2].copy()          # c_2, c_4, ..., c_{2n}
    x = np.exp(np.linspace(0.0, np.log(1.0 / k), grid))
    t = x * x
    R = x.copy()
    for l in range(n):
        R *= (t + c_num[l]) / (t + c_den[l])
    d0 = 2.0 / (R.max() + R.min())
    delta = float(np.max(np.abs(1.0 - d0 * R)))
    a = np.empty(n)
    for l in range(n):
        num = np.prod(c_num - c_den[l])
        den = np.prod(np.delete(c_den, l) - c_den[l])
        a[l] = num / den
    return {"k": k, "n": n, "d0": d0, "a": a, "c_den": c_den, "c_num": c_num, "delta": delta}


def rational_sign_scalar(lam, co, lam_min):
    """Scalar approximant of sign(lam) from the partial-fraction form."""
    x = np.asarray(lam, dtype=float) / lam_min
    t = x * x
    s = np.ones_like(t)
    for a, c in zip(co["a"], co["c_den"]):
        s = s + a / (t + c)
    return co["d0"] * x * s


def rational_sign_product(lam, co, lam_min):
    """Same approximant from the product form (independent evaluation)."""
    x = np.asarray(lam, dtype=float) / lam_min
    t = x * x
    R = x.copy()
    for cn_, cd_ in zip(co["c_num"], co["c_den"]):
        R = R * (t + cn_) / (t + cd_)
    return co["d0"] * R

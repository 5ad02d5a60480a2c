"""ctypes front end of the plain-C sparse oracle (sparse.c) and its build step.

Test infrastructure only. build() compiles sparse.c with gcc and OpenMP into
oracle/_build/libo2.so; every call converts arrays to contiguous complex128.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparse.c")
_OUT = os.path.join(_HERE, "_build", "libo2.so")
_lib = None


def build(force=False):
    """Compile sparse.c (gcc -O2 -fopenmp); returns the library path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", _OUT, "-lm"])
    return _OUT


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        P = ctypes.c_void_p
        I_ = ctypes.c_int
        D = ctypes.c_double
        L.o2_wilson.argtypes = [P, P, P, P, D, I_]
        L.o2_gamma5.argtypes = [P, P, ctypes.c_long]
        L.o2_q2_shift.argtypes = [P, P, P, P, D, I_, D, P]
        L.o2_cg_shift.argtypes = [P, P, P, P, D, I_, D, D, I_]
        L.o2_cg_shift.restype = I_
        L.o2_sign_zolo.argtypes = [P, P, P, P, D, I_, D, D, I_, P, P, D, I_, P]
        L.o2_sign_zolo.restype = I_
        L.o2_overlap.argtypes = [P, P, P, P, D, I_, D, D, D, I_, P, P, D, I_, P]
        L.o2_overlap.restype = I_
        L.o2_threads.restype = I_
        L.o2_gamma5_diag.argtypes = [P]
        _lib = L
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def threads():
    return lib().o2_threads()


def gamma5_diag():
    out = np.zeros(4)
    lib().o2_gamma5_diag(_p(out))
    return out


def wilson(psi, U, dims, m0, antiperiodic=True):
    psi, U, d = _c(psi), _c(U), _dims(dims)
    out = np.empty_like(psi)
    lib().o2_wilson(_p(out), _p(psi), _p(U), _p(d), float(m0), int(antiperiodic))
    return out


def q2_shift(psi, U, dims, m0, sigma=0.0, antiperiodic=True):
    psi, U, d = _c(psi), _c(U), _dims(dims)
    out = np.empty_like(psi)
    tmp = np.empty_like(psi)
    lib().o2_q2_shift(_p(out), _p(psi), _p(U), _p(d), float(m0), int(antiperiodic),
                      float(sigma), _p(tmp))
    return out


def cg_shift(b, U, dims, m0, sigma, tol, maxit=100000, antiperiodic=True):
    b, U, d = _c(b), _c(U), _dims(dims)
    x = np.empty_like(b)
    it = lib().o2_cg_shift(_p(x), _p(b), _p(U), _p(d), float(m0), int(antiperiodic),
                           float(sigma), float(tol), int(maxit))
    return x, it


def sign_zolo(b, U, dims, m0, lam_min, co, tol, maxit=100000, antiperiodic=True):
    """sign(Q) b with Zolotarev coefficients `co` (see zolotarev.py)."""
    b, U, d = _c(b), _c(U), _dims(dims)
    out = np.empty_like(b)
    a = np.ascontiguousarray(co["a"], dtype=np.float64)
    c = np.ascontiguousarray(co["c_den"], dtype=np.float64)
    iters = np.zeros(len(a), dtype=np.int32)
    st = lib().o2_sign_zolo(_p(out), _p(b), _p(U), _p(d), float(m0), int(antiperiodic),
                            float(lam_min), float(co["d0"]), len(a), _p(a), _p(c),
                            float(tol), int(maxit), _p(iters))
    if st != 0:
        raise RuntimeError("oracle CG did not converge")
    return out, iters


def overlap(b, U, dims, m0, rho, lam_min, co, tol, maxit=100000, antiperiodic=True):
    """D_N b = rho b + Gamma5 sign(Q) b."""
    b, U, d = _c(b), _c(U), _dims(dims)
    out = np.empty_like(b)
    a = np.ascontiguousarray(co["a"], dtype=np.float64)
    c = np.ascontiguousarray(co["c_den"], dtype=np.float64)
    iters = np.zeros(len(a), dtype=np.int32)
    st = lib().o2_overlap(_p(out), _p(b), _p(U), _p(d), float(m0), int(antiperiodic),
                          float(rho), float(lam_min), float(co["d0"]), len(a), _p(a), _p(c),
                          float(tol), int(maxit), _p(iters))
    if st != 0:
        raise RuntimeError("oracle CG did not converge")
    return out, iters

"""Host-only checks of the C-ABI library: it builds, loads without a GPU,
exports every function include/ovl.h declares, its Python struct mirrors match the C layout,
and its host-side Zolotarev
coefficients (own AGM/Landen elliptic functions) match the oracle's
(scipy elliptic functions, grid-centred scale)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1410_7170_gb300 as ovl
from oracle import zolotarev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1410_7170_gb300 import build
    build.build()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(?:ovl_status|const char \*)\s*(\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol():
    decl = _declared()
    assert {"ovl_create", "wilson_apply", "sign_apply", "ovl_apply", "ovl_solve", "ovl_destroy"} <= decl
    out = subprocess.run(["nm", "-D", "--defined-only", ovl.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s(\w+)$", out, flags=re.M))
    assert decl <= exported, decl - exported
    L = ovl.lib()
    for name in decl:
        assert hasattr(L, name)


def test_params_default_are_paper_values():
    """Table 2 / Table 3 defaults (see tests/golden/paper_values.json)."""
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))
    p = ovl.params_default()
    assert p.tol_outer == gold["table2_eps_outer"]["value"]
    assert p.restart == gold["table2_restart"]["value"]
    assert p.relax_factor == gold["table2_relaxation_factor"]["value"]
    assert p.eps_prec == gold["table2_eps_prec"]["value"]
    assert p.eps_inner == gold["table3_eps_inner_prec"]["value"]
    assert p.restart_inner == gold["table3_restart_inner"]["value"]


@pytest.mark.parametrize("k,n", [(0.05, 20), (0.01, 20), (0.1, 5), (0.2, 3), (0.003, 30)])
def test_host_zolotarev_matches_oracle(k, n):
    d0, a, c, delta = ovl.ovl_zolotarev(k, n)
    co = zolotarev.zolotarev_coefficients(k, n)
    assert np.allclose(c, co["c_den"], rtol=1e-11)
    assert np.allclose(a, co["a"], rtol=1e-9, atol=1e-14 * np.abs(co["a"]).max())
    assert abs(d0 - co["d0"]) < 1e-12 * co["d0"] + co["delta"]
    lam = np.exp(np.linspace(0, np.log(1 / k), 20001))
    approx = d0 * lam * (1 + sum(ai / (lam ** 2 + ci) for ai, ci in zip(a, c)))
    assert np.max(np.abs(1 - approx)) <= max(delta, 1e-14) * 1.01 + 1e-14


def test_zolotarev_rejects_bad_interval():
    with pytest.raises(ovl.OvlError):
        ovl.ovl_zolotarev(1.5, 10)
    with pytest.raises(ovl.OvlError):
        ovl.ovl_zolotarev(0.1, 0)


@pytest.mark.parametrize("n", [1, 3, 17, 96])
def test_host_hermitian_eig_matches_numpy(n):
    """The host eigensolver (Rayleigh-Ritz steps of the low-mode eigensolver): the
    eigenvalues agree with LAPACK's, the eigenvectors satisfy A Z = Z diag(w) and are
    orthonormal."""
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.conj().T
    w, Z = ovl.hermitian_eig(A)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * np.abs(w).max()
    assert np.abs(A @ Z - Z * w).max() < 1e-12 * np.abs(w).max()
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() < 1e-13


def _eig_ok(A, tol=1e-13):
    w, Z = ovl.hermitian_eig(A)
    n = A.shape[0]
    sc = max(np.abs(w).max(), 1e-300)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() <= tol * sc * 10
    assert np.abs(A @ Z - Z * w).max() <= tol * sc * 10
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= tol * 10
    assert np.all(np.diff(w) >= 0)


def test_host_hermitian_eig_structured_cases():
    """Shapes the solvers produce: the thick-restart projected matrix (diagonal block of
    kept Ritz values, bordered by one complex row and column, then tridiagonal), clustered
    and repeated eigenvalues, a graded spectrum over 13 decades, a tridiagonal matrix whose
    couplings underflow, 2 x 2, and the zero matrix."""
    rng = np.random.default_rng(11)
    n, kk = 40, 8
    H = np.zeros((n, n), complex)
    H[np.arange(kk), np.arange(kk)] = rng.uniform(0.3, 1.0, kk)
    H[kk, :kk] = rng.normal(size=kk) + 1j * rng.normal(size=kk)
    H[:kk, kk] = H[kk, :kk].conj()
    for j in range(kk, n):
        H[j, j] = rng.uniform(1.0, 50.0)
    for j in range(kk, n - 1):
        H[j + 1, j] = H[j, j + 1] = rng.uniform(0.1, 5.0)
    _eig_ok(H)
    W, _ = np.linalg.qr(rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30)))
    _eig_ok((W * np.repeat([1.0, 1.0 + 1e-12, 2.0, 5.0, -3.0], 6)) @ W.conj().T)
    W, _ = np.linalg.qr(rng.normal(size=(25, 25)) + 1j * rng.normal(size=(25, 25)))
    _eig_ok((W * np.logspace(-10, 3, 25)) @ W.conj().T)
    T = np.diag(np.arange(10.0)) + np.diag(np.full(9, 1e-300), 1) + np.diag(np.full(9, 1e-300), -1)
    _eig_ok(T.astype(complex))
    _eig_ok(np.array([[1.0, 2 - 1j], [2 + 1j, -3.0]]))
    w, Z = ovl.hermitian_eig(np.zeros((5, 5), complex))
    assert np.all(w == 0) and np.allclose(Z.conj().T @ Z, np.eye(5))


def test_host_hermitian_eig_degenerate_and_diagonal():
    w, Z = ovl.hermitian_eig(np.diag([3.0, 1.0, 1.0, -2.0]).astype(complex))
    assert np.allclose(w, [-2.0, 1.0, 1.0, 3.0])
    with pytest.raises(ovl.OvlError):
        ovl.hermitian_eig(np.zeros((0, 0), dtype=complex))


def test_request_bytes_estimate_covers_options():
    """The serving loop's admission estimate (host only) grows by the Krylov sign basis and
    the deflation vectors when those options are on, scales with the volume, and rejects
    bad requests."""
    dims = (16, 16, 16, 16)
    v64 = 24 * 16 ** 4 * 8
    base = ovl.request_bytes(dims)
    kry = ovl.request_bytes(dims, params=ovl.params_default(sign_method=ovl.OVL_SIGN_KRYLOV, krylov_m=40,
                                                            krylov_keep=8))
    assert kry - base >= (40 + 8 + 3) * v64
    defl = ovl.request_bytes(dims, params=ovl.params_default(n_deflate=16))
    assert defl - base >= (2 * 16 + 1) * v64 + (66 + 33 + 2) * v64
    assert ovl.request_bytes((32, 32, 32, 32)) > 15 * base
    assert ovl.request_bytes(dims, n_rhs=4) > base
    with pytest.raises(ovl.OvlError):
        ovl.request_bytes((0, 4, 4, 4))


def test_binding_structs_match_the_c_abi(tmp_path):
    """Every ctypes mirror of an ovl.h struct has the C struct's size and each field the C
    offset (compiled from include/ovl.h with the host C compiler): a field added on one side
    only would otherwise shift every later field silently."""
    mirrors = [ovl.ovl_params, ovl.ovl_stats, ovl.ovl_request, ovl.ovl_result, ovl.ovl_prof_kernel, ovl.ovl_prof]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ovl.h"', "int main(void) {"]
    for m in mirrors:
        name = m.__name__
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in m._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for m in mirrors:
        name = m.__name__
        assert int(got[name]) == ctypes.sizeof(m), name
        for f in m._fields_:
            assert int(got["%s.%s" % (name, f[0])]) == getattr(m, f[0]).offset, (name, f[0])

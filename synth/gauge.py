"""Seeded SU(3) gauge fields: random links, stout smearing, gauge rotations.

The random links follow the recipe U = exp(i*eps*H) with H a traceless
Hermitian 3x3 matrix drawn from complex Gaussian entries. Stout smearing
follows Eq. (stout) and Eq. (Zdef) of Sec. 4, read with the sign that makes
one step lower the Wilson gauge action (Sec. 4 states that it does; with the
plaquette Q = staple * U^H as defined in Eq. (plaquette_def1) that requires
Z = +1/2 (M - M^H) - 1/6 tr(M - M^H) I). All links of one step are updated
in parallel from the previous field (the Lie-Euler step of Sec. 4).
"""

import numpy as np


def _lattice_view(U, dims):
    L0, L1, L2, L3 = dims
    return U.reshape(L0, L1, L2, L3, 4, 3, 3)


def _expi_hermitian(H, eps):
    """exp(i*eps*H) for a stack of Hermitian 3x3 matrices via eigh."""
    w, W = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ab,...b,...cb->...ac", W, ph, W.conj())


def random_su3(shape, eps, rng):
    """Stack of SU(3) matrices exp(i*eps*H), H traceless Hermitian.

    H = (A + A^H)/2 - tr/3 I with A having i.i.d. complex Gaussian entries
    (real and imaginary parts ~ N(0,1)), drawn as re then im in C order.
    """
    shape = tuple(shape)
    re = rng.standard_normal(shape + (3, 3))
    im = rng.standard_normal(shape + (3, 3))
    A = re + 1j * im
    H = 0.5 * (A + np.swapaxes(A.conj(), -1, -2))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    return _expi_hermitian(H, eps)


def stout_step(U, dims, eps):
    """One stout step U -> exp(eps Z) U for every link (Eqs. stout, Zdef)."""
    Uf = _lattice_view(U, dims)
    out = np.empty_like(Uf)

    def fwd(F, nu):      # F(x + nu-hat)
        return np.roll(F, -1, axis=nu)

    def bwd(F, nu):      # F(x - nu-hat)
        return np.roll(F, 1, axis=nu)

    def dag(A):
        return np.swapaxes(A.conj(), -1, -2)

    for mu in range(4):
        Umu = Uf[..., mu, :, :]
        M = np.zeros_like(Umu)
        for nu in range(4):
            if nu == mu:
                continue
            Unu = Uf[..., nu, :, :]
            # Q^{mu,nu}_x = U_nu(x) U_mu(x+nu) U_nu(x+mu)^H U_mu(x)^H
            M += Unu @ fwd(Umu, nu) @ dag(fwd(Unu, mu)) @ dag(Umu)
            # Q^{mu,-nu}_x = U_nu(x-nu)^H U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^H
            Unu_b = bwd(Unu, nu)
            M += dag(Unu_b) @ bwd(Umu, nu) @ fwd(Unu_b, mu) @ dag(Umu)
        B = 0.5 * (M - dag(M))
        tr = np.trace(B, axis1=-2, axis2=-1) / 3.0
        Z = B - tr[..., None, None] * np.eye(3)
        # Z is anti-Hermitian traceless: Z = i*Hz with Hz = -i Z Hermitian
        Hz = -1j * Z
        Hz = 0.5 * (Hz + dag(Hz))
        out[..., mu, :, :] = _expi_hermitian(Hz, eps) @ Umu
    return out.reshape(U.shape)


def stout_smear(U, dims, eps, steps):
    for _ in range(steps):
        U = stout_step(U, dims, eps)
    return U


def gauge_field(dims, eps, seed, stout_steps=0, stout_eps=0.1, device=None):
    """Seeded gauge field [V][4][3][3] complex128 (numpy).

    Links exp(i*eps*H) drawn site-major (site, then direction), then
    `stout_steps` stout steps with parameter `stout_eps`. With device (e.g.
    "cuda") the staples and the exponentials (scaling and squaring of a Taylor
    series instead of eigh) are evaluated in torch FP64 on that device; the
    random draws are the same numpy draws, so the two paths agree to ~1e-14.
    """
    dims = tuple(int(d) for d in dims)
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    if device is not None:
        return _gauge_field_torch(dims, V, eps, rng, stout_steps, stout_eps, device)
    U = random_su3((V, 4), eps, rng)
    if stout_steps:
        U = stout_smear(U, dims, stout_eps, stout_steps)
    return np.ascontiguousarray(U)


def _gauge_field_torch(dims, V, eps, rng, stout_steps, stout_eps, device):
    import torch
    re = rng.standard_normal((V, 4, 3, 3))
    im = rng.standard_normal((V, 4, 3, 3))
    A = torch.complex(torch.from_numpy(re), torch.from_numpy(im)).to(device)
    del re, im
    eye = torch.eye(3, dtype=torch.complex128, device=device)

    def dag(X):
        return X.conj().transpose(-1, -2)

    def expi(H, e):
        # exp(i e H) by scaling and squaring: Taylor series of exp(A / 2^s) to order 16,
        # then s squarings; s makes max ||A||_F / 2^s <= 1/4 (series error ~ 1e-20)
        A = (1j * e) * H
        nrm = float(torch.linalg.matrix_norm(A).max())
        sc = 0
        while nrm / (1 << sc) > 0.25:
            sc += 1
        A = A / float(1 << sc)
        out = eye.expand_as(A).clone()
        term = eye.expand_as(A).clone()
        for k in range(1, 17):
            term = term @ A / k
            out = out + term
        for _ in range(sc):
            out = out @ out
        return out

    H = 0.5 * (A + dag(A))
    tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1).real / 3.0
    H = H - tr[..., None, None] * eye
    del A
    U = expi(H, eps).reshape(tuple(dims) + (4, 3, 3))
    del H
    for _ in range(stout_steps):
        out = torch.empty_like(U)
        for mu in range(4):
            Umu = U[..., mu, :, :]
            M = torch.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = U[..., nu, :, :]
                M += Unu @ torch.roll(Umu, -1, nu) @ dag(torch.roll(Unu, -1, mu)) @ dag(Umu)
                Unu_b = torch.roll(Unu, 1, nu)
                M += dag(Unu_b) @ torch.roll(Umu, 1, nu) @ torch.roll(Unu_b, -1, mu) @ dag(Umu)
            B = 0.5 * (M - dag(M))
            trb = torch.diagonal(B, dim1=-2, dim2=-1).sum(-1) / 3.0
            Z = B - trb[..., None, None] * eye
            Hz = -1j * Z
            Hz = 0.5 * (Hz + dag(Hz))
            out[..., mu, :, :] = expi(Hz, stout_eps) @ Umu
            del M, B, Z, Hz
        U = out
    return np.ascontiguousarray(U.reshape(V, 4, 3, 3).cpu().numpy())


def random_gauge_rotation(dims, seed, eps=np.pi):
    """One SU(3) matrix per site, [V][3][3], for gauge-covariance checks."""
    V = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    return random_su3((V,), eps, rng)


def gauge_transform_links(U, dims, G):
    """U'_mu(x) = G(x) U_mu(x) G(x + mu-hat)^H."""
    L0, L1, L2, L3 = dims
    Uf = _lattice_view(U, dims)
    Gf = G.reshape(L0, L1, L2, L3, 3, 3)
    out = np.empty_like(Uf)
    for mu in range(4):
        Gn = np.roll(Gf, -1, axis=mu)
        out[..., mu, :, :] = Gf @ Uf[..., mu, :, :] @ np.swapaxes(Gn.conj(), -1, -2)
    return out.reshape(U.shape)


def gauge_transform_spinor(psi, G):
    """psi'(x) = G(x) psi(x) on the colour index; psi is [..., V, 4, 3]."""
    return np.einsum("vab,...vsb->...vsa", G, psi)

"""Discretised Green's operators of the 2-D TM problem (Sec. 2.1, Eq. 1-4).

Conventions (readings, the paper states only the integrals):
  * time factor e^{-i w t}; scalar Green's function g(r, r') = (i/4) H0^(1)(k0 |r - r'|),
    so physical media have Re chi >= 0, Im chi >= 0 as assumed below Eq. (7);
  * pulse basis on the M1 x M2 grid, each square cell replaced by the disk of equal
    area, radius a (Richmond's method).  Integrating k0^2 g over such a disk gives
      off-diagonal  G[m, n] = (i pi k0 a / 2) J1(k0 a) H0^(1)(k0 rho_mn)
      diagonal      G[n, n] = (i pi k0 a / 2) H1^(1)(k0 a) - 1
    using  int_0^a H0(k0 rho) rho d rho = (k0 a H1(k0 a) + 2i/pi) / k0^2.
  * G_S (Eq. 2, receivers outside the DOI) uses the off-diagonal formula.
  * incident field of transmitter p: line source H0^(1)(k0 |r - r_p|) normalised to unit
    magnitude at the DOI centre, or a unit plane wave exp(i k0 d_p . r).

Pinned by: Mie series of a homogeneous cylinder (tests/test_oracle_physics.py), reciprocity
of the full-aperture data, dense == FFT application, adjoint identities.
"""
from __future__ import annotations

import numpy as np
from scipy import fft as sfft
from scipy import special

from .problem import Problem


def richmond_coeffs(p: Problem):
    """(c_off, c_self): G_D[m,n] = c_off * H0(k0 rho) off the diagonal, G_D[n,n] = c_self."""
    ka = p.k0 * p.a_eq
    c = 1j * np.pi * ka / 2.0
    return c * special.j1(ka), c * special.hankel1(1, ka) - 1.0


def gd_dense(p: Problem) -> np.ndarray:
    """Dense G_D as an [M][M] complex128 matrix over the flattened [y][x] grid (Eq. 3)."""
    X, Y = p.centres()
    x, y = X.ravel(), Y.ravel()
    rho = np.hypot(x[:, None] - x[None, :], y[:, None] - y[None, :])
    c_off, c_self = richmond_coeffs(p)
    np.fill_diagonal(rho, 1.0)                      # placeholder, overwritten below
    G = c_off * special.hankel1(0, p.k0 * rho)
    np.fill_diagonal(G, c_self)
    return G


def gd_circulant_kernel(p: Problem) -> np.ndarray:
    """Block-Toeplitz kernel of G_D embedded in a (2 M2) x (2 M1) circulant: [2ny][2nx].

    Entry [dy mod 2ny][dx mod 2nx] holds G_D between cells separated by (dx, dy) pixels,
    |dx| < nx, |dy| < ny; the rows/columns at offset exactly ny / nx are zero.
    """
    c_off, c_self = richmond_coeffs(p)
    Py, Px = 2 * p.ny, 2 * p.nx
    ox = np.arange(Px)
    oy = np.arange(Py)
    ox = np.where(ox < p.nx, ox, ox - Px).astype(float)          # signed x offsets
    oy = np.where(oy < p.ny, oy, oy - Py).astype(float)
    DX, DY = np.meshgrid(ox * p.dx, oy * p.dy)
    rho = np.hypot(DX, DY)
    rho[0, 0] = 1.0
    g = c_off * special.hankel1(0, p.k0 * rho)
    g[0, 0] = c_self
    g[p.ny, :] = 0.0
    g[:, p.nx] = 0.0
    return g


def gd_spectrum(p: Problem) -> np.ndarray:
    """2-D DFT of the circulant kernel (scipy's FFT as a library primitive)."""
    return sfft.fft2(gd_circulant_kernel(p))


def gd_apply(p: Problem, J: np.ndarray, adjoint: bool = False, spec: np.ndarray = None) -> np.ndarray:
    """G_D J (or G_D^H J) for J of shape [..., ny, nx] via zero-padded FFT convolution.

    G_D is symmetric (its kernel depends on |r - r'| only) so G_D^H = conj(G_D), applied
    with the conjugated spectrum of the (even) circulant kernel.
    """
    if spec is None:
        spec = gd_spectrum(p)
    if adjoint:
        spec = np.conj(spec)
    Py, Px = 2 * p.ny, 2 * p.nx
    pad = np.zeros(J.shape[:-2] + (Py, Px), dtype=np.complex128)
    pad[..., :p.ny, :p.nx] = J
    out = sfft.ifft2(spec * sfft.fft2(pad))
    return out[..., :p.ny, :p.nx]


def gs_dense(p: Problem) -> np.ndarray:
    """Receiver operator G_S as [nr][M] complex128 (Eq. 2, 4)."""
    X, Y = p.centres()
    x, y = X.ravel(), Y.ravel()
    rho = np.hypot(p.rx[:, 0:1] - x[None, :], p.rx[:, 1:2] - y[None, :])
    c_off, _ = richmond_coeffs(p)
    return c_off * special.hankel1(0, p.k0 * rho)


def einc(p: Problem) -> np.ndarray:
    """Incident fields [ni][ny][nx] complex128 on the cell centres."""
    X, Y = p.centres()
    if p.inc_kind == 0:
        out = np.empty((p.ni, p.ny, p.nx), dtype=np.complex128)
        for t in range(p.ni):
            tx, ty = p.tx[t]
            rho = np.hypot(X - tx, Y - ty)
            norm = abs(special.hankel1(0, p.k0 * np.hypot(tx, ty)))
            out[t] = special.hankel1(0, p.k0 * rho) / norm
        return out
    d = p.tx / np.linalg.norm(p.tx, axis=1, keepdims=True)
    return np.exp(1j * p.k0 * (d[:, 0, None, None] * X[None] + d[:, 1, None, None] * Y[None]))


def einc_at(p: Problem, pts: np.ndarray) -> np.ndarray:
    """Incident fields of every transmitter at arbitrary points pts [n][2]: [ni][n]."""
    if p.inc_kind == 0:
        out = np.empty((p.ni, pts.shape[0]), dtype=np.complex128)
        for t in range(p.ni):
            tx, ty = p.tx[t]
            rho = np.hypot(pts[:, 0] - tx, pts[:, 1] - ty)
            out[t] = special.hankel1(0, p.k0 * rho) / abs(special.hankel1(0, p.k0 * np.hypot(tx, ty)))
        return out
    d = p.tx / np.linalg.norm(p.tx, axis=1, keepdims=True)
    return np.exp(1j * p.k0 * (d @ pts.T))


class Operators:
    """The fixed operators of one geometry, assembled once: G_D spectrum, G_S, E_inc."""

    def __init__(self, p: Problem, dense_gd: bool = False):
        self.p = p
        self.spec = gd_spectrum(p)
        self.GS = gs_dense(p)
        self.Einc = einc(p)
        self.GD = gd_dense(p) if dense_gd else None

    def gd(self, J, adjoint=False):
        if self.GD is not None:
            flat = J.reshape(J.shape[:-2] + (-1,))
            G = self.GD.conj() if adjoint else self.GD         # symmetric => G^H = conj(G)
            return (flat @ G.T).reshape(J.shape)
        return gd_apply(self.p, J, adjoint, self.spec)

    def gs(self, J):
        """[..., ny, nx] -> [..., nr]"""
        return J.reshape(J.shape[:-2] + (-1,)) @ self.GS.T

    def gsh(self, d):
        """G_S^H: [..., nr] -> [..., ny, nx]"""
        out = d @ self.GS.conj()
        return out.reshape(d.shape[:-1] + (self.p.ny, self.p.nx))

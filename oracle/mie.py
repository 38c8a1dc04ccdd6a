"""Bessel-series scattered field of a homogeneous circular cylinder (independent pin).

Not in the paper: this is the textbook closed form used to pin the oracle's Green's
operators and forward solve (Eq. 1-5) from outside the oracle.  A cylinder of
radius a centred on the origin, relative permittivity eps_r (complex for lossy
media, e^{-i w t}), illuminated by the line source H0^(1)(k0 |r - r_s|) normalised to
unit magnitude at the origin.  With n_r = sqrt(eps_r), k1 = n_r k0, matching E_z and
dE_z/drho at rho = a gives the exterior coefficient

    a_n = [n_r J_n'(k1 a) J_n(k0 a) - J_n'(k0 a) J_n(k1 a)]
          / [J_n(k1 a) H_n'(k0 a) - n_r J_n'(k1 a) H_n(k0 a)]

and, by Graf's addition theorem H0(k0|r - r_s|) = sum_n J_n(k0 rho) H_n(k0 rho_s) e^{in(phi - phi_s)}
(rho < rho_s), the scattered field at rho > a

    E_sca(rho, phi) = sum_n a_n H_n(k0 rho_s) H_n(k0 rho) e^{in(phi - phi_s)} / |H0(k0 rho_s)|.

Pinned by energy conservation (tests/test_oracle_physics.py): every partial wave of a lossless
cylinder has |1 + 2 a_n| = 1, and a lossy one (Im eps_r > 0) absorbs, |1 + 2 a_n| < 1.
"""
from __future__ import annotations

import numpy as np
from scipy import special


def mie_coeffs(k0: float, radius: float, eps_r: complex, nmax: int) -> np.ndarray:
    n = np.arange(-nmax, nmax + 1)
    nr = np.sqrt(complex(eps_r))
    k1 = nr * k0
    x0, x1 = k0 * radius, k1 * radius
    Jn0, dJn0 = special.jv(n, x0), special.jvp(n, x0)
    Jn1, dJn1 = special.jv(n, x1), special.jvp(n, x1)
    Hn0, dHn0 = special.hankel1(n, x0), special.h1vp(n, x0)
    return (nr * dJn1 * Jn0 - dJn0 * Jn1) / (Jn1 * dHn0 - nr * dJn1 * Hn0)


def mie_esca_line_source(k0: float, radius: float, eps_r: complex, src: np.ndarray, rx: np.ndarray,
                         nmax: int = None) -> np.ndarray:
    """Scattered field [ni][nr] for sources src [ni][2] and receivers rx [nr][2]."""
    if nmax is None:
        nmax = int(np.ceil(abs(np.sqrt(complex(eps_r))) * k0 * radius)) + 25
    an = mie_coeffs(k0, radius, eps_r, nmax)
    n = np.arange(-nmax, nmax + 1)
    rs, ps = np.hypot(src[:, 0], src[:, 1]), np.arctan2(src[:, 1], src[:, 0])
    rr, pr = np.hypot(rx[:, 0], rx[:, 1]), np.arctan2(rx[:, 1], rx[:, 0])
    Hs = special.hankel1(n[None, :], k0 * rs[:, None])            # [ni][n]
    Hr = special.hankel1(n[None, :], k0 * rr[:, None])            # [nr][n]
    ph = np.exp(1j * n[None, None, :] * (pr[None, :, None] - ps[:, None, None]))
    out = np.einsum("in,rn,irn->ir", an[None, :] * Hs, Hr, ph)
    return out / np.abs(special.hankel1(0, k0 * rs))[:, None]

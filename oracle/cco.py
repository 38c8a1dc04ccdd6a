"""Contrast-compensated operator (Sec. 2.4, Eq. 10, 11) and its adjoint, float64.

Test infrastructure: only tests/, the smoke check and the benchmark's CPU baseline use the oracle.

  box_mean          mean over the (2r+1)^2 window clipped to the grid (divided by the in-bounds count)
  guided_self       self-guided filter G(I | I) of a real image (He et al.; guide = input)
  gain              eta = eta_max sigmoid((|chi| - tau) / delta) and d eta / d|chi|      (Eq. 11)
  cco               chi_CCO = (1 + eta) G(chi | chi) + eta chi                            (Eq. 10)
  cco_vjp           the cotangent on chi of <c, chi_CCO(chi)> (the CCO's adjoint), hand-derived

Readings (the paper cites the guided filter but prints no radius, regulariser or complex rule):
box radius 2 with windows clipped to the grid, eps = 1e-2, Re and Im filtered separately, eta from
|chi|, and Eq. (10) taken as printed (weights 1 + eta and +eta).  When the CCO sits inside the loss
(Problem.cco_in_loss), the regularisers of Eq. (17)-(19) act on chi_CCO and the gradient runs
back through cco_vjp.

Gradient convention (PyTorch's, as in loss.py): for real L and complex z, g = dL/dRe z + i dL/dIm z;
cco_vjp(chi, c) returns that g for L = sum Re(conj(c) chi_CCO), i.e. c given in the same convention.

The adjoint follows the forward's steps in reverse.  For one real channel I, with windows w(k)
of n_k pixels:
  mu_k = box(I)_k, var_k = box(I^2)_k - mu_k^2, a_k = var_k / (var_k + eps), b_k = mu_k (1 - a_k),
  q_i  = box(a)_i I_i + box(b)_i;
and box's adjoint sends c_i to every pixel k of w(i) with weight 1 / n_i.

Pinned by tests/test_oracle_cco.py: box's adjoint against the transpose of the box matrix built
from unit images, central differences of the filter, of the whole CCO and of the loss with the CCO
inside it, the eps -> inf limit (the adjoint of the double box mean, from that matrix) and the
eps -> 0 limit (the identity).
"""
from __future__ import annotations

import numpy as np


def box_mean(a: np.ndarray, r: int) -> np.ndarray:
    """Mean over the (2r+1)^2 window clipped to the grid (divided by the in-bounds count)."""
    ny, nx = a.shape
    out = np.zeros_like(a)
    for i in range(ny):
        i0, i1 = max(0, i - r), min(ny, i + r + 1)
        for j in range(nx):
            j0, j1 = max(0, j - r), min(nx, j + r + 1)
            out[i, j] = a[i0:i1, j0:j1].mean()
    return out


def box_mean_adjoint(c: np.ndarray, r: int) -> np.ndarray:
    """Adjoint of box_mean: each c[i] spread over the window of i, divided by that window's count."""
    ny, nx = c.shape
    out = np.zeros_like(c)
    for i in range(ny):
        i0, i1 = max(0, i - r), min(ny, i + r + 1)
        for j in range(nx):
            j0, j1 = max(0, j - r), min(nx, j + r + 1)
            out[i0:i1, j0:j1] += c[i, j] / ((i1 - i0) * (j1 - j0))
    return out


def guided_self(I: np.ndarray, r: int, eps: float) -> np.ndarray:
    """Self-guided filter G(I | I) of a real image (He et al., guide = input)."""
    mu = box_mean(I, r)
    var = box_mean(I * I, r) - mu * mu
    a = var / (var + eps)
    b = mu - a * mu
    return box_mean(a, r) * I + box_mean(b, r)


def guided_self_vjp(I: np.ndarray, c: np.ndarray, r: int, eps: float) -> np.ndarray:
    """d/dI of sum(c * guided_self(I)) for a real image I and a real cotangent c."""
    mu = box_mean(I, r)
    var = box_mean(I * I, r) - mu * mu
    a = var / (var + eps)
    # q = box(a) I + box(b)
    c_I = box_mean(a, r) * c
    c_a = box_mean_adjoint(c * I, r)
    c_b = box_mean_adjoint(c, r)
    # b = mu - a mu
    c_mu = c_b * (1.0 - a)
    c_a = c_a - c_b * mu
    # a = var / (var + eps)
    c_var = c_a * eps / (var + eps) ** 2
    # var = box(I^2) - mu^2, mu = box(I)
    c_mu = c_mu - 2.0 * mu * c_var
    return c_I + 2.0 * I * box_mean_adjoint(c_var, r) + box_mean_adjoint(c_mu, r)


def gain(mag: np.ndarray, eta_max: float, tau: float, delta: float):
    """eta = eta_max sigmoid((|chi| - tau) / delta) (Eq. 11) and its derivative in |chi|."""
    sg = 1.0 / (1.0 + np.exp(-(mag - tau) / delta))
    return eta_max * sg, eta_max * sg * (1.0 - sg) / delta


def cco(chi: np.ndarray, r: int = 2, eps: float = 1e-2, eta_max: float = 0.1, tau: float = 3.0,
        delta: float = 0.5, unsharp: bool = False) -> np.ndarray:
    """chi_CCO = (1 + eta) G(chi|chi) + eta chi, eta = eta_max sigmoid((|chi| - tau)/delta)  (Eq. 10, 11)."""
    g = guided_self(chi.real, r, eps) + 1j * guided_self(chi.imag, r, eps)
    eta, _ = gain(np.abs(chi), eta_max, tau, delta)
    return (1.0 + eta) * g + (-eta if unsharp else eta) * chi


def cco_vjp(chi: np.ndarray, c: np.ndarray, r: int = 2, eps: float = 1e-2, eta_max: float = 0.1,
            tau: float = 3.0, delta: float = 0.5, unsharp: bool = False) -> np.ndarray:
    """Cotangent on chi of sum Re(conj(c) cco(chi)) (both in PyTorch's complex convention)."""
    sgn = -1.0 if unsharp else 1.0
    g = guided_self(chi.real, r, eps) + 1j * guided_self(chi.imag, r, eps)
    mag = np.abs(chi)
    eta, deta = gain(mag, eta_max, tau, delta)
    # out = (1 + eta) g + sgn eta chi: through g (each channel through its own filter) ...
    c_g = (1.0 + eta) * c
    c_chi = guided_self_vjp(chi.real, c_g.real, r, eps) + 1j * guided_self_vjp(chi.imag, c_g.imag, r, eps)
    # ... directly ...
    c_chi = c_chi + sgn * eta * c
    # ... and through eta(|chi|), d|chi| / d(Re, Im) = chi / |chi| (0 at chi = 0)
    c_eta = np.real(np.conj(c) * (g + sgn * chi))
    unit = np.where(mag > 0, chi / np.where(mag > 0, mag, 1.0), 0.0)
    return c_chi + c_eta * deta * unit

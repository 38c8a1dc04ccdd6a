"""Initialisation, outer optimisation and post-processing of a PDF solve, float64.

  bp_init     back-propagation contrast chi_(0) and R_(0) = beta chi / (beta chi + 1)   (Sec. 3.1, Eq. 7)
  csi_step    alpha_(0) = one gradient step of L^CSI from alpha = 0 at fixed R_(0)     (Sec. 3.1, Eq. 12)
  adam        torch.optim.Adam semantics on (Re, Im) pairs, lr 1e-2                     (Sec. 3.3)
  cco         contrast-compensated operator with a self-guided filter (oracle/cco.py)   (Sec. 2.4, Eq. 10, 11)
  relerr      ||chi - chi_true|| / ||chi_true||
  pdf_solve   the whole reconstruction: init, Adam loop on L, final chi, CCO

Readings (the paper cites but does not print them):
  * BP: J_p = gamma_p G_S^H E_sca,p with gamma_p = ||G_S^H E_p||^2 / ||G_S G_S^H E_p||^2 (the
    scale minimising ||E_p - gamma G_S G_S^H E_p||); E_tot = E_inc + G_D J; chi_(0) is the per-pixel
    least-squares fit of J = chi E_tot over all incidences.
  * CSI step size: the exact minimiser along -grad of the quadratic L^CSI at fixed R_(0),
    t = ||g||^2 / (2 sum_w c_w ||M_w g||^2).
  * Guided filter (He et al.): guide = input, box radius 2 normalised by the in-bounds
    count, eps = 1e-2, applied to Re and Im separately; eta from |chi|; Eq. (10) taken as printed.

Pinned by: Adam against torch.optim.Adam, line-search optimality, guided-filter limits
(eps -> 0 gives the identity, eps -> inf the double box mean, constants pass through).
pdf_solve is pinned as a composition: its first Adam step lowers L at the rate ||g||_1 (Re and
Im parts) as lr -> 0, which a conjugated gradient or a reversed step breaks; started from the
exact coefficients of the true currents (K = M, no noise, no regularisers) it returns the true
contrast after a step bounded by lr max|g| / eps.  The RelErr a whole solve reaches on a given
workload has no printed value in the paper to compare with.
"""
from __future__ import annotations

import numpy as np

from . import fbe
from .cco import box_mean, cco, guided_self  # noqa: F401  (the CCO of the final output)
from .green import Operators
from .loss import chi_from_R, loss_grad, forward, norms


def bp_init(ops: Operators, esca: np.ndarray):
    """Return (chi0 [ny][nx], R0 [ny][nx], J_bp [ni][ny][nx])."""
    p = ops.p
    gh = ops.gsh(esca)                                  # G_S^H E_p
    ggh = ops.gs(gh)                                    # G_S G_S^H E_p
    num = np.sum(np.abs(gh.reshape(p.ni, -1)) ** 2, axis=1)
    den = np.sum(np.abs(ggh) ** 2, axis=1)
    gamma = num / den
    Jbp = gamma[:, None, None] * gh
    Etot = ops.Einc + ops.gd(Jbp)
    chi0 = np.sum(Jbp * np.conj(Etot), axis=0) / np.sum(np.abs(Etot) ** 2, axis=0)
    R0 = p.beta * chi0 / (p.beta * chi0 + 1.0)
    return chi0, R0, Jbp


def csi_step(ops: Operators, esca: np.ndarray, R0: np.ndarray) -> np.ndarray:
    """alpha_(0) = -t g, g = grad of L^CSI (Eq. 12) at alpha = 0 with R fixed to R0."""
    p = ops.p
    beta = p.beta
    ein2, esc2 = norms(ops, esca)
    # residuals at alpha = 0
    rd0 = -esca
    r0 = R0[None] * ops.Einc
    gJ = (2.0 / esc2) * ops.gsh(rd0) \
        + (2.0 / ein2) * (np.conj(beta) * (np.conj(R0)[None] * r0 - r0) + ops.gd(np.conj(R0)[None] * r0, adjoint=True))
    g = fbe.analysis(gJ, p.ky, p.kx)
    Jg = fbe.synth(g, p.ny, p.nx)
    m1 = ops.gs(Jg)
    m2 = R0[None] * (beta * Jg + ops.gd(Jg)) - beta * Jg
    den = np.sum(np.abs(m1) ** 2) / esc2 + np.sum(np.abs(m2) ** 2) / ein2
    t = np.sum(np.abs(g) ** 2) / (2.0 * den)
    return -t * g


def csi_loss(ops, esca, R0, alpha):
    """L^CSI of Eq. (12) at fixed R0 (used by the line-search pin)."""
    p = ops.p
    ein2, esc2 = norms(ops, esca)
    J = fbe.synth(alpha, p.ny, p.nx)
    r = R0[None] * (ops.Einc + ops.gd(J)) - p.beta * (1.0 - R0[None]) * J
    rd = ops.gs(J) - esca
    return float(np.sum(np.abs(rd) ** 2) / esc2 + np.sum(np.abs(r) ** 2) / ein2)


class Adam:
    """torch.optim.Adam (no weight decay, no amsgrad) on the real view of a complex array."""

    def __init__(self, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = None
        self.v = None
        self.t = 0

    def step(self, x: np.ndarray, g: np.ndarray) -> np.ndarray:
        xr = np.stack([x.real, x.imag], -1)
        gr = np.stack([g.real, g.imag], -1)
        if self.m is None:
            self.m = np.zeros_like(xr)
            self.v = np.zeros_like(xr)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * gr
        self.v = self.b2 * self.v + (1 - self.b2) * gr * gr
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        xr = xr - self.lr * mh / (np.sqrt(vh) + self.eps)
        return xr[..., 0] + 1j * xr[..., 1]


def relerr(chi: np.ndarray, chi_true: np.ndarray) -> float:
    return float(np.linalg.norm(chi - chi_true) / np.linalg.norm(chi_true))


def final_chi(ops, esca, alpha):
    return forward(ops, esca, alpha).chi


def pdf_solve(ops: Operators, esca: np.ndarray, iters: int, lr: float = 1e-2, alpha0=None,
              chi_true=None, apply_cco: bool = True, history: bool = False):
    """Whole reconstruction; returns dict(alpha, chi, chi_cco, relerr, relerr_cco, losses)."""
    if alpha0 is None:
        _, R0, _ = bp_init(ops, esca)
        alpha0 = csi_step(ops, esca, R0)
    alpha = alpha0.copy()
    opt = Adam(lr=lr)
    losses = []
    for _ in range(iters):
        terms, g = loss_grad(ops, esca, alpha)
        if history:
            losses.append(terms)
        alpha = opt.step(alpha, g)
    chi = final_chi(ops, esca, alpha)
    out = dict(alpha=alpha, alpha0=alpha0, chi=chi, losses=np.array(losses))
    p = ops.p
    out["chi_cco"] = cco(chi, p.cco_radius, p.cco_eps, p.cco_eta_max, p.cco_tau, p.cco_delta) if apply_cco else chi
    if chi_true is not None:
        out["relerr"] = relerr(chi, chi_true)
        out["relerr_cco"] = relerr(out["chi_cco"], chi_true)
    return out

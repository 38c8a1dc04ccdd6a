"""Composite PDF loss and its hand-derived gradient, float64 (Sec. 3.2, Eq. 6, 7, 13-19).

Forward, for coefficients alpha [ni][ky][kx]:
  J_p   = F*_T(alpha_p)                                   (Eq. 9)
  s_p   = beta J_p + E_inc,p + G_D J_p                     (bracket of Eq. 6)
  R_n   = sum_p beta J_p,n conj(s_p,n) / sum_p |s_p,n|^2   (reading: R-hat is the per-pixel
                                                            least-squares solution of Eq. 6)
  chi_n = R_n / (beta (1 - R_n))                           (inverse of Eq. 7, |1 - R| clamped)
  r_p   = R E_inc,p + [R G_D - beta (I - R)] J_p  = R s_p - beta J_p     (Eq. 15)
  L_State  = sum_p ||r_p||^2 / ||E_inc||^2                 (Eq. 15)
  L_Data   = sum_p ||G_S J_p - E_sca,p||^2 / ||E_sca||^2   (Eq. 16)
  L_Bound  = || ReLU(-Re chi) ||^2                         (Eq. 17)
  L_TV     = sum sqrt(|chi_{i,j+1}-chi_{i,j}|^2 + |chi_{i+1,j}-chi_{i,j}|^2 + eps_tv)   (Eq. 18)
  L_Bridge = sum sigmoid((|chi|-tau_B)/tau_B) exp(-|grad|chi||^2)                    (Eq. 19)
  L = L_State + L_Data + lam1 L_Bound + lam2 L_TV + lam3 L_Bridge                   (Eq. 13, 14)
With Problem.cco_in_loss the three regularisers act on chi_CCO = (1 + eta) G(chi|chi) + eta chi
(Eq. 10, 11; oracle/cco.py) instead of chi, and their cotangent returns to chi through the CCO's
adjoint before it continues to R and J.

Readings: differences are forward differences in pixel units, a difference
that would leave the grid is zero; |chi| = sqrt(|chi|^2 + eps_abs).

Gradient convention (PyTorch's for a real function of complex z):
g = dL/dRe z + i dL/dIm z.  Since R minimises L_State pixel by pixel, the
derivative of L_State through R vanishes (envelope theorem); the regularisers
reach J through chi(R(J)) and that path is differentiated in full.

Pinned by: the CIE identity at the exact forward solution (L_State = 0 and
R = R_true when nothing is truncated), closed forms of the regularisers,
the envelope identity, and central finite differences of L itself
(tests/test_oracle_loss.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cco as ccomod
from . import fbe
from .green import Operators


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _fdiff(a):
    """Forward differences along x and y with zero where the neighbour is off-grid."""
    gx = np.zeros_like(a)
    gy = np.zeros_like(a)
    gx[:, :-1] = a[:, 1:] - a[:, :-1]
    gy[:-1, :] = a[1:, :] - a[:-1, :]
    return gx, gy


def _fdiff_adjoint(cx, cy):
    """Adjoint of _fdiff: returns sum over terms of c * d(difference)/d(pixel)."""
    out = np.zeros_like(cx)
    out[:, 1:] += cx[:, :-1]
    out[:, :-1] -= cx[:, :-1]
    out[1:, :] += cy[:-1, :]
    out[:-1, :] -= cy[:-1, :]
    return out


def chi_from_R(R: np.ndarray, beta: complex, q_min: float):
    """chi = R / (beta (1 - R)) with |1 - R| clamped to q_min; returns (chi, clamped mask)."""
    q = 1.0 - R
    aq = np.abs(q)
    clamped = aq < q_min
    qs = np.where(clamped, q_min * np.where(aq > 0, q / np.where(aq > 0, aq, 1.0), 1.0), q)
    return R / (beta * qs), clamped


def reg_terms(p, chi: np.ndarray):
    """(L_Bound, L_TV, L_Bridge) and the cotangent c_chi of lam1 L_Bound + lam2 L_TV + lam3 L_Bridge."""
    # Eq. (17)
    neg = np.maximum(-chi.real, 0.0)
    l_bound = float(np.sum(neg * neg))
    c_bound = -2.0 * neg + 0j
    # Eq. (18)
    dx, dy = _fdiff(chi)
    t = np.sqrt(np.abs(dx) ** 2 + np.abs(dy) ** 2 + p.eps_tv)
    l_tv = float(np.sum(t))
    c_tv = _fdiff_adjoint(dx / t, dy / t)
    # Eq. (19)
    mag = np.sqrt(np.abs(chi) ** 2 + p.eps_abs)
    gx, gy = _fdiff(mag)
    sg = _sigmoid((mag - p.tau_b) / p.tau_b)
    e = np.exp(-(gx * gx + gy * gy))
    l_bridge = float(np.sum(sg * e))
    dmag = sg * (1.0 - sg) / p.tau_b * e + _fdiff_adjoint(-2.0 * gx * sg * e, -2.0 * gy * sg * e)
    c_bridge = dmag * chi / mag
    c = p.lam_bound * c_bound + p.lam_tv * c_tv + p.lam_bridge * c_bridge
    return (l_bound, l_tv, l_bridge), c


@dataclass
class Forward:
    J: np.ndarray
    GJ: np.ndarray
    s: np.ndarray
    N: np.ndarray
    D: np.ndarray
    R: np.ndarray
    chi: np.ndarray
    clamped: np.ndarray
    chi_reg: np.ndarray         # the image the regularisers act on: chi, or chi_CCO with cco_in_loss
    r: np.ndarray
    rd: np.ndarray
    terms: np.ndarray           # [L, State, Data, Bound, TV, Bridge]


def norms(ops: Operators, esca: np.ndarray):
    return float(np.sum(np.abs(ops.Einc) ** 2)), float(np.sum(np.abs(esca) ** 2))


def forward(ops: Operators, esca: np.ndarray, alpha: np.ndarray) -> Forward:
    p = ops.p
    beta = p.beta
    J = fbe.synth(alpha, p.ny, p.nx)
    GJ = ops.gd(J)
    s = beta * J + ops.Einc + GJ
    N = np.sum(beta * J * np.conj(s), axis=0)
    D = np.sum(np.abs(s) ** 2, axis=0)
    R = N / D
    chi, clamped = chi_from_R(R, beta, p.q_min)
    r = R[None] * s - beta * J
    rd = ops.gs(J) - esca
    ein2, esc2 = norms(ops, esca)
    l_state = float(np.sum(np.abs(r) ** 2)) / ein2
    l_data = float(np.sum(np.abs(rd) ** 2)) / esc2
    chi_reg = ccomod.cco(chi, p.cco_radius, p.cco_eps, p.cco_eta_max, p.cco_tau, p.cco_delta) \
        if p.cco_in_loss else chi
    (lb, ltv, lbr), _ = reg_terms(p, chi_reg)
    total = l_state + l_data + p.lam_bound * lb + p.lam_tv * ltv + p.lam_bridge * lbr
    return Forward(J, GJ, s, N, D, R, chi, clamped, chi_reg, r, rd,
                   np.array([total, l_state, l_data, lb, ltv, lbr]))


def loss(ops, esca, alpha) -> np.ndarray:
    return forward(ops, esca, alpha).terms


def loss_grad(ops: Operators, esca: np.ndarray, alpha: np.ndarray):
    """Return (terms[6], grad_alpha) with grad in PyTorch's complex convention."""
    p = ops.p
    beta = p.beta
    bc = np.conj(beta)
    f = forward(ops, esca, alpha)
    ein2, esc2 = norms(ops, esca)

    # Regulariser cotangent on chi, pulled back to R through chi = R / (beta (1 - R)):
    # d chi / d R = 1 / (beta (1 - R)^2) (holomorphic), zero where the clamp is active.
    _, c_chi = reg_terms(p, f.chi_reg)
    if p.cco_in_loss:
        c_chi = ccomod.cco_vjp(f.chi, c_chi, p.cco_radius, p.cco_eps, p.cco_eta_max, p.cco_tau, p.cco_delta)
    dchi_dR = 1.0 / (beta * (1.0 - f.R) ** 2)
    c_R = np.where(f.clamped, 0.0, np.conj(dchi_dR) * c_chi)
    # R = N / D with N = sum beta J conj(s), D = sum |s|^2:  w = c_R / D
    w = c_R / f.D
    c_s = np.conj(w)[None] * beta * f.J - 2.0 * np.real(np.conj(w) * f.R)[None] * f.s

    # L_State with R held fixed: A = diag(R)(beta I + G_D) - beta I,  grad = 2/||Einc||^2 A^H r
    u = (2.0 / ein2) * np.conj(f.R)[None] * f.r + c_s                     # goes through G_D^H
    v = (2.0 / ein2) * (-bc * (1.0 - np.conj(f.R)))[None] * f.r \
        + bc * (w[None] * f.s + c_s)                                        # pointwise part
    gJ = v + ops.gd(u, adjoint=True) + (2.0 / esc2) * ops.gsh(f.rd)
    return f.terms, fbe.analysis(gJ, p.ky, p.kx)

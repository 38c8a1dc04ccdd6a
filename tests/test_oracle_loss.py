"""Pins of the oracle's loss (Eq. 13-19) and gradient.

CIE identity at the exact forward solution, closed forms of the regularisers,
the envelope identity of the least-squares R, and central finite differences.
"""
import numpy as np
import pytest

import scenes
from oracle import fbe, loss
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import Problem, from_workload


def _setup(n=16, ni=4, nr=8, k=5, dense=True, **kw):
    w = scenes.workload("c1", nx=n, ny=n, ni=ni, nr=nr, kx=k, ky=k)
    p = from_workload(w, **kw)
    ops = Operators(p, dense_gd=dense)
    chi = scenes.rasterise([scenes.Shape("disk", 0.1, 0.0, 0.45, eps_r=2.5, tan_d=0.2)], n, n, 2.0)
    J, _, esca = forward_solve(ops, chi)
    return p, ops, chi, J, esca


def test_cie_identity_at_exact_solution():
    # With no truncation (K = M) and alpha = F_T(J_true): R-hat = R_true, chi-hat = chi_true,
    # and both physics residuals vanish (Eq. 6, 15, 16).
    p, ops, chi, J, esca = _setup(k=16)
    f = loss.forward(ops, esca, fbe.analysis(J, 16, 16))
    r_true = p.beta * chi / (p.beta * chi + 1)
    assert np.abs(f.R - r_true).max() < 1e-12
    assert np.abs(f.chi - chi).max() < 1e-12
    assert f.terms[1] < 1e-24 and f.terms[2] < 1e-24


def test_state_loss_equals_lippmann_schwinger_form():
    # R E_inc + [R G_D - beta (I - R)] J  ==  R s - beta J  for arbitrary R (algebra of Eq. 15)
    p, ops, chi, J, esca = _setup()
    rng = np.random.default_rng(3)
    a = rng.standard_normal((p.ni, 5, 5)) + 1j * rng.standard_normal((p.ni, 5, 5))
    f = loss.forward(ops, esca, a)
    Jt = f.J
    direct = f.R[None] * ops.Einc + f.R[None] * ops.gd(Jt) - p.beta * (1 - f.R[None]) * Jt
    assert np.abs(direct - f.r).max() < 1e-12 * np.abs(direct).max()


def test_envelope_least_squares_R():
    p, ops, chi, J, esca = _setup()
    rng = np.random.default_rng(4)
    a = rng.standard_normal((p.ni, 5, 5)) + 1j * rng.standard_normal((p.ni, 5, 5))
    f = loss.forward(ops, esca, a)
    # stationarity: sum_p (R s - beta J) conj(s) = 0 at every pixel
    assert np.abs(np.sum(f.r * np.conj(f.s), axis=0)).max() < 1e-12 * np.abs(f.N).max()
    # and L_State grows under any perturbation of R
    base = np.sum(np.abs(f.r) ** 2)
    for _ in range(3):
        dR = 1e-3 * (rng.standard_normal(f.R.shape) + 1j * rng.standard_normal(f.R.shape))
        assert np.sum(np.abs((f.R + dR)[None] * f.s - p.beta * f.J) ** 2) > base


def _p(nx=5, ny=4):
    return Problem(nx=nx, ny=ny, side_x=1.0, side_y=1.0, k0=2 * np.pi, tx=np.zeros((1, 2)),
                   rx=np.zeros((1, 2)), kx=1, ky=1)


def test_regulariser_closed_forms():
    p = _p()
    m = p.nx * p.ny
    c = 0.7 - 0.2j
    (lb, ltv, lbr), _ = loss.reg_terms(p, np.full((4, 5), c))
    assert lb == 0.0
    assert abs(ltv - m * np.sqrt(p.eps_tv)) < 1e-15
    assert abs(lbr - m / (1 + np.exp(-(abs(c) - p.tau_b) / p.tau_b))) < 1e-9
    # all-negative real part: L_Bound = M c^2
    (lb, _, _), _ = loss.reg_terms(p, np.full((4, 5), -0.3 + 1j))
    assert abs(lb - m * 0.09) < 1e-12
    # vertical step of height h between columns 1 and 2: one x-difference per row
    h = 2.0
    step = np.zeros((4, 5), complex)
    step[:, 2:] = h
    (_, ltv, _), _ = loss.reg_terms(p, step)
    assert abs(ltv - (4 * np.sqrt(h * h + p.eps_tv) + (m - 4) * np.sqrt(p.eps_tv))) < 1e-12
    # linear ramp chi = g * x: |grad| = g except the last column
    g = 0.3
    ramp = np.tile(g * np.arange(5.0), (4, 1)).astype(complex)
    (_, ltv, _), _ = loss.reg_terms(p, ramp)
    assert abs(ltv - (16 * np.sqrt(g * g + p.eps_tv) + 4 * np.sqrt(p.eps_tv))) < 1e-12
    # bridge at |chi| = tau_B on a constant image: M / 2
    (_, _, lbr), _ = loss.reg_terms(p, np.full((4, 5), p.tau_b + 0j))
    assert abs(lbr - m / 2) < 1e-9


def test_regulariser_brute_force_tiny():
    # pure-Python loops over the pixel sums of Eq. (18) and (19) on a 3 x 3 image
    p = _p(3, 3)
    rng = np.random.default_rng(5)
    chi = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))

    def at(i, j):
        return chi[i][j] if (0 <= i < 3 and 0 <= j < 3) else None
    tv = 0.0
    br = 0.0
    for i in range(3):
        for j in range(3):
            dx = (at(i, j + 1) - at(i, j)) if at(i, j + 1) is not None else 0.0
            dy = (at(i + 1, j) - at(i, j)) if at(i + 1, j) is not None else 0.0
            tv += np.sqrt(abs(dx) ** 2 + abs(dy) ** 2 + p.eps_tv)
            m0 = np.sqrt(abs(at(i, j)) ** 2 + p.eps_abs)
            mx = np.sqrt(abs(at(i, j + 1)) ** 2 + p.eps_abs) - m0 if at(i, j + 1) is not None else 0.0
            my = np.sqrt(abs(at(i + 1, j)) ** 2 + p.eps_abs) - m0 if at(i + 1, j) is not None else 0.0
            br += 1 / (1 + np.exp(-(m0 - p.tau_b) / p.tau_b)) * np.exp(-(mx * mx + my * my))
    (_, ltv, lbr), _ = loss.reg_terms(p, chi)
    assert abs(ltv - tv) < 1e-12 and abs(lbr - br) < 1e-12


@pytest.mark.parametrize("weights", [(1e-3, 1e-5, 1e-5), (1.0, 0.3, 0.5)])
def test_gradient_central_differences(weights):
    p, ops, chi, J, esca = _setup(dense=False)
    p.lam_bound, p.lam_tv, p.lam_bridge = weights
    rng = np.random.default_rng(6)
    a = 0.3 * (rng.standard_normal((p.ni, 5, 5)) + 1j * rng.standard_normal((p.ni, 5, 5)))
    _, g = loss.loss_grad(ops, esca, a)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
        fd = (loss.loss(ops, esca, a + h * d)[0] - loss.loss(ops, esca, a - h * d)[0]) / (2 * h)
        an = np.sum(np.real(np.conj(g) * d))
        assert abs(fd - an) < 1e-7 * max(abs(an), 1e-3)


def test_gradient_of_each_component_by_differences():
    # single-coordinate differences on Re and Im of a few coefficients (checks the convention
    # g = dL/dRe + i dL/dIm, not just directional consistency)
    p, ops, chi, J, esca = _setup(dense=False)
    rng = np.random.default_rng(7)
    a = 0.3 * (rng.standard_normal((p.ni, 5, 5)) + 1j * rng.standard_normal((p.ni, 5, 5)))
    _, g = loss.loss_grad(ops, esca, a)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (3, 4, 1)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            e = np.zeros_like(a)
            e[idx] = unit
            fd = (loss.loss(ops, esca, a + h * e)[0] - loss.loss(ops, esca, a - h * e)[0]) / (2 * h)
            assert abs(fd - part(g[idx])) < 1e-7 * max(abs(g).max(), 1e-3)


def test_terms_at_zero_coefficients():
    # alpha = 0: J = 0, so s = E_inc and the least-squares R-hat is 0 (Eq. 6), r = 0 and
    # L_State = 0 (Eq. 15); r_d = -E_sca, so L_Data = ||E_sca||^2 / ||E_sca||^2 = 1 exactly (Eq. 16);
    # chi-hat = 0 gives L_Bound = 0, L_TV = M sqrt(eps_TV) and L_Bridge = M sigmoid((sqrt(eps_abs)
    # - tau_B) / tau_B) (Eq. 17-19, all differences zero); L is their weighted sum (Eq. 13).
    p, ops, chi, J, esca = _setup()
    t = loss.forward(ops, esca, np.zeros((p.ni, p.ky, p.kx), complex)).terms
    m = p.nx * p.ny
    assert t[1] == 0.0 and abs(t[2] - 1.0) < 1e-15 and t[3] == 0.0
    assert abs(t[4] - m * np.sqrt(p.eps_tv)) < 1e-15
    br = m / (1.0 + np.exp(-(np.sqrt(p.eps_abs) - p.tau_b) / p.tau_b))
    assert abs(t[5] - br) < 1e-12 * br
    assert abs(t[0] - (1.0 + p.lam_tv * t[4] + p.lam_bridge * t[5])) < 1e-15

"""Planted mistakes in the oracle (CPU only) must be caught by the pins.

Each test patches one plausible error into the oracle -- a dropped term, a wrong
sign, a non-conjugated adjoint -- and checks that the pin it should trip does trip.
"""
import numpy as np
import pytest

import scenes
from oracle import green, loss
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.mie import mie_esca_line_source
from oracle.problem import from_workload


def _mie_err(n=32):
    p = from_workload(scenes.workload("c1", nx=n, ny=n, ni=6, nr=10))
    ops = Operators(p, dense_gd=True)
    chi = scenes.rasterise([scenes.Shape("disk", 0.0, 0.0, 0.4, eps_r=2.0)], n, n, 2.0)
    _, _, esca = forward_solve(ops, chi)
    r_eq = np.sqrt(np.count_nonzero(chi) * p.dx * p.dy / np.pi)
    ref = mie_esca_line_source(p.k0, r_eq, 2.0, p.tx, p.rx)
    return np.linalg.norm(esca - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("mistake", ["drop_minus_one", "h0_instead_of_h1", "conj_kernel"])
def test_green_mistakes_break_mie(monkeypatch, mistake):
    good = green.richmond_coeffs

    def bad(p):
        c_off, c_self = good(p)
        ka = p.k0 * p.a_eq
        if mistake == "drop_minus_one":
            return c_off, c_self + 1.0
        if mistake == "h0_instead_of_h1":
            from scipy import special
            return c_off, 1j * np.pi * ka / 2 * special.hankel1(0, ka) - 1.0
        return np.conj(c_off), np.conj(c_self)
    assert _mie_err() < 0.08
    monkeypatch.setattr(green, "richmond_coeffs", bad)
    assert _mie_err() > 0.08


def test_adjoint_without_conjugate_breaks_finite_differences(monkeypatch):
    p = from_workload(scenes.workload("c1", nx=12, ny=12, ni=3, nr=6, kx=5, ky=5))
    ops = Operators(p)
    chi = scenes.rasterise([scenes.Shape("disk", 0.0, 0.0, 0.4, eps_r=2.0)], 12, 12, 2.0)
    _, _, esca = forward_solve(ops, chi)
    rng = np.random.default_rng(0)
    a = 0.3 * (rng.standard_normal((3, 5, 5)) + 1j * rng.standard_normal((3, 5, 5)))
    d = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)

    def mismatch():
        _, g = loss.loss_grad(ops, esca, a)
        h = 1e-6
        fd = (loss.loss(ops, esca, a + h * d)[0] - loss.loss(ops, esca, a - h * d)[0]) / (2 * h)
        return abs(fd - np.sum(np.real(np.conj(g) * d))) / abs(fd)
    assert mismatch() < 1e-7
    orig = ops.gd
    monkeypatch.setattr(ops, "gd", lambda J, adjoint=False: orig(J, False))
    assert mismatch() > 1e-3


def _first_step_rate():
    """(L(alpha_0) - L(alpha_1)) / lr of the oracle solve at small lr, and ||g||_1 at alpha_0."""
    from oracle import solve
    p = from_workload(scenes.workload("c1", nx=12, ny=12, ni=3, nr=6, kx=5, ky=5))
    ops = Operators(p, dense_gd=True)
    chi = scenes.rasterise([scenes.Shape("disk", 0.0, 0.0, 0.4, eps_r=2.0)], 12, 12, 2.0)
    _, _, esca = forward_solve(ops, chi)
    rng = np.random.default_rng(1)
    a0 = 0.2 * (rng.standard_normal((3, 5, 5)) + 1j * rng.standard_normal((3, 5, 5)))
    _, g = loss.loss_grad(ops, esca, a0)
    lr = 1e-6
    out = solve.pdf_solve(ops, esca, 2, lr=lr, alpha0=a0, apply_cco=False, history=True)
    return (out["losses"][0, 0] - out["losses"][1, 0]) / lr, np.abs(g.real).sum() + np.abs(g.imag).sum()


@pytest.mark.parametrize("mistake", ["conjugated_gradient", "ascent"])
def test_solve_mistakes_break_first_step_descent(monkeypatch, mistake):
    from oracle import solve
    rate, l1 = _first_step_rate()
    assert abs(rate - l1) < 2e-2 * l1
    if mistake == "conjugated_gradient":
        good = solve.loss_grad
        monkeypatch.setattr(solve, "loss_grad", lambda o, e, a: (lambda t, g: (t, np.conj(g)))(*good(o, e, a)))
    else:
        good_step = solve.Adam.step
        monkeypatch.setattr(solve.Adam, "step", lambda self, x, g: 2 * x - good_step(self, x, g))
    rate, l1 = _first_step_rate()
    assert abs(rate - l1) > 0.1 * l1


def test_mie_mistakes_break_energy_pins(monkeypatch):
    # H^(2) in place of H^(1) (the e^{+i w t} convention) turns the lossy cylinder into a gain
    # medium; a sign error in a_n breaks lossless unitarity.
    from scipy import special
    from oracle import mie
    good = mie.mie_coeffs

    def lossless_err():
        return np.abs(np.abs(1 + 2 * mie.mie_coeffs(2 * np.pi, 0.4, 3.5, 30)) - 1).max()

    def lossy_gain():
        return np.abs(1 + 2 * mie.mie_coeffs(2 * np.pi, 0.4, 2.5 * (1 + 0.3j), 30)).max()
    assert lossless_err() < 1e-10 and lossy_gain() <= 1 + 1e-12
    fake = type("special", (), {"jv": special.jv, "jvp": special.jvp,
                                "hankel1": special.hankel2, "h1vp": special.h2vp})
    monkeypatch.setattr(mie, "special", fake)
    assert lossy_gain() > 1.01
    monkeypatch.setattr(mie, "special", special)
    monkeypatch.setattr(mie, "mie_coeffs", lambda *a: -good(*a))
    assert lossless_err() > 1e-2


def _periodic_fdiff(a):
    return np.roll(a, -1, axis=1) - a, np.roll(a, -1, axis=0) - a


def _adjoint_without_outflow(cx, cy):
    out = np.zeros_like(cx)
    out[:, 1:] += cx[:, :-1]
    out[1:, :] += cy[:-1, :]
    return out


@pytest.mark.parametrize("mistake", ["periodic_differences", "flipped_sigmoid", "half_adjoint"])
def test_regulariser_mistakes_break_their_pins(monkeypatch, mistake):
    # Eq. 17-19: each plant must fail the pin that guards it: the closed forms of the regularisers
    # on constant, step and ramp images (boundary and sigmoid direction), or the central
    # differences of the loss with heavy regulariser weights (the adjoint of the differences).
    from tests import test_oracle_loss as pins
    if mistake == "periodic_differences":
        monkeypatch.setattr(loss, "_fdiff", _periodic_fdiff)
        check = pins.test_regulariser_closed_forms
    elif mistake == "flipped_sigmoid":
        monkeypatch.setattr(loss, "_sigmoid", lambda x: 1.0 / (1.0 + np.exp(x)))
        check = pins.test_regulariser_closed_forms
    else:
        monkeypatch.setattr(loss, "_fdiff_adjoint", _adjoint_without_outflow)
        check = lambda: pins.test_gradient_central_differences((1.0, 0.3, 0.5))   # noqa: E731
    with pytest.raises(AssertionError):
        check()


@pytest.mark.parametrize("mistake", ["floor_half_set", "unnormalised_synthesis", "analysis_with_inverse_dft"])
def test_fbe_mistakes_break_their_pins(monkeypatch, mistake):
    # Eq. 9: a mode set shifted by one for odd K, a synthesis without the unitary 1/sqrt(M), and an
    # analysis that uses the inverse DFT (the conjugate basis) each fail the brute-force basis sums
    # or the adjoint / left-inverse identities.
    from oracle import fbe
    from tests import test_oracle_fbe as pins
    good_synth = fbe.synth
    if mistake == "floor_half_set":
        monkeypatch.setattr(fbe, "mode_indices",
                            lambda K, M: np.array([j if j < K // 2 else M - K + j for j in range(K)]))
    elif mistake == "unnormalised_synthesis":
        monkeypatch.setattr(fbe, "synth", lambda a, ny, nx: good_synth(a, ny, nx) * np.sqrt(ny * nx))
    else:
        def bad_analysis(J, ky, kx):
            ny, nx = J.shape[-2:]
            iy, ix = fbe.mode_indices(ky, ny), fbe.mode_indices(kx, nx)
            return np.fft.ifft2(J, norm="ortho")[..., iy[:, None], ix[None, :]]
        monkeypatch.setattr(fbe, "analysis", bad_analysis)
    failed = 0
    for check in (lambda: pins.test_synth_is_sum_of_basis_functions(6, 8, 3, 5),
                  pins.test_analysis_is_adjoint_and_left_inverse):
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed >= 1


@pytest.mark.parametrize("mistake", ["chi_with_1_plus_R", "swapped_norms"])
def test_cie_and_normalisation_mistakes_break_their_pins(monkeypatch, mistake):
    # Eq. 7 read as chi = R / (beta (1 + R)) fails the CIE identity at the exact solution; the
    # incident and measured norms swapped (Eq. 15, 16) fail L_Data = 1 at zero coefficients.
    from tests import test_oracle_loss as pins
    if mistake == "chi_with_1_plus_R":
        monkeypatch.setattr(loss, "chi_from_R", lambda R, beta, q_min: (R / (beta * (1.0 + R)), np.zeros(R.shape, bool)))
        check = pins.test_cie_identity_at_exact_solution
    else:
        good = loss.norms
        monkeypatch.setattr(loss, "norms", lambda ops, esca: good(ops, esca)[::-1])
        check = pins.test_terms_at_zero_coefficients
    with pytest.raises(AssertionError):
        check()


def _cco_fd_mismatch():
    from oracle import cco
    rng = np.random.default_rng(3)
    chi = rng.uniform(0.0, 5.0, (9, 8)) * np.exp(1j * rng.uniform(-0.4, 1.2, (9, 8)))
    c = rng.standard_normal(chi.shape) + 1j * rng.standard_normal(chi.shape)
    d = rng.standard_normal(chi.shape) + 1j * rng.standard_normal(chi.shape)
    h = 1e-6
    f = lambda z: np.sum(np.real(np.conj(c) * cco.cco(z, eps=0.05)))
    fd = (f(chi + h * d) - f(chi - h * d)) / (2 * h)
    an = np.sum(np.real(np.conj(cco.cco_vjp(chi, c, eps=0.05)) * d))
    return abs(fd - an) / abs(fd)


def test_cco_adjoint_without_gain_derivative_breaks_differences(monkeypatch):
    from oracle import cco
    assert _cco_fd_mismatch() < 1e-8
    good = cco.gain
    # the forward keeps its gain, the adjoint loses d eta / d|chi|
    monkeypatch.setattr(cco, "gain", lambda m, e, t, dl: (good(m, e, t, dl)[0], 0.0 * m))
    assert _cco_fd_mismatch() > 1e-4


def test_cco_adjoint_variance_factor_breaks_differences(monkeypatch):
    from oracle import cco

    def bad_vjp(I, c, r, eps):                 # the var = box(I^2) - mu^2 path without its factor 2
        mu = cco.box_mean(I, r)
        var = cco.box_mean(I * I, r) - mu * mu
        a = var / (var + eps)
        c_I = cco.box_mean(a, r) * c
        c_a = cco.box_mean_adjoint(c * I, r)
        c_b = cco.box_mean_adjoint(c, r)
        c_mu = c_b * (1.0 - a)
        c_a = c_a - c_b * mu
        c_var = c_a * eps / (var + eps) ** 2
        c_mu = c_mu - mu * c_var
        return c_I + I * cco.box_mean_adjoint(c_var, r) + cco.box_mean_adjoint(c_mu, r)
    assert _cco_fd_mismatch() < 1e-8
    monkeypatch.setattr(cco, "guided_self_vjp", bad_vjp)
    assert _cco_fd_mismatch() > 1e-4


def test_box_adjoint_with_the_receivers_count_breaks_the_transpose(monkeypatch):
    from oracle import cco
    from tests.test_oracle_cco import box_matrix

    def bad(c, r):                              # divides by the count of the window around k, not i
        ny, nx = c.shape
        out = np.zeros_like(c)
        for i in range(ny):
            for j in range(nx):
                i0, i1 = max(0, i - r), min(ny, i + r + 1)
                j0, j1 = max(0, j - r), min(nx, j + r + 1)
                out[i, j] = c[i0:i1, j0:j1].sum() / ((i1 - i0) * (j1 - j0))
        return out
    B = box_matrix(6, 7, 2)
    c = np.random.default_rng(0).standard_normal((6, 7))
    assert np.abs(cco.box_mean_adjoint(c, 2).ravel() - B.T @ c.ravel()).max() < 1e-14
    monkeypatch.setattr(cco, "box_mean_adjoint", bad)
    assert np.abs(cco.box_mean_adjoint(c, 2).ravel() - B.T @ c.ravel()).max() > 1e-3

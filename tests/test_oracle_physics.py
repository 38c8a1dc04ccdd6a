"""Pins of the oracle's Green's operators and forward solve (Eq. 1-5) against outside facts.

None of these re-types an oracle formula: each compares against a closed form
(Mie series, Graf's addition theorem integrated by quadrature), a symmetry the
physics fixes (reciprocity), or the Born limit.
"""
import numpy as np
import pytest
from scipy import integrate, special

import scenes
from oracle.forward import forward_solve
from oracle.green import Operators, gd_apply, gd_dense, richmond_coeffs
from oracle.mie import mie_esca_line_source
from oracle.problem import Problem, from_workload


def _disk_problem(n, ni=6, nr=10, side=2.0, radius=5.0, dense=None):
    w = scenes.workload("c1", nx=n, ny=n, side=side, ni=ni, nr=nr, radius=radius)
    p = from_workload(w)
    return p, Operators(p, dense_gd=(n <= 32) if dense is None else dense)


def _mie_error(n, eps_r, r=0.4):
    p, ops = _disk_problem(n)
    shape = scenes.Shape("disk", 0.0, 0.0, r, eps_r=eps_r.real, tan_d=eps_r.imag / eps_r.real)
    chi = scenes.rasterise([shape], n, n, p.side_x)
    _, _, esca = forward_solve(ops, chi)
    r_eq = np.sqrt(np.count_nonzero(chi) * p.dx * p.dy / np.pi)   # equal-area radius of the staircase disk
    ref = mie_esca_line_source(p.k0, r_eq, eps_r, p.tx, p.rx)
    return np.linalg.norm(esca - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("eps_r", [2.0 + 0j, 2.5 + 0.5j])
def test_mie_series_convergence(eps_r):
    e16, e32, e64 = (_mie_error(n, eps_r) for n in (16, 32, 64))
    assert e32 < 0.08 and e64 < 0.03
    assert e64 < e32 < e16


def test_richmond_self_term_by_quadrature():
    # diagonal of G_D = k0^2 (i/4) int_disk H0(k0 rho) dA over the equal-area disk (Eq. 1)
    p, _ = _disk_problem(16)
    k0, a = p.k0, p.a_eq
    re = integrate.quad(lambda t: special.j0(k0 * t) * 2 * np.pi * t, 0, a, limit=200)[0]
    im = integrate.quad(lambda t: special.y0(k0 * t) * 2 * np.pi * t, 0, a, limit=200)[0]
    ref = k0 ** 2 * 0.25j * (re + 1j * im)
    _, c_self = richmond_coeffs(p)
    assert abs(c_self - ref) < 1e-9 * abs(ref)


def test_richmond_off_diagonal_by_quadrature():
    # Graf: int_disk H0(k0 |r - r'|) dA' = (2 pi a / k0) J1(k0 a) H0(k0 rho); check by 2-D quadrature
    p, _ = _disk_problem(16)
    k0, a, rho = p.k0, p.a_eq, 3.0 * p.dx

    def f(t, ph, part):
        d = np.sqrt(rho ** 2 + t ** 2 - 2 * rho * t * np.cos(ph))
        return (special.j0 if part == 0 else special.y0)(k0 * d) * t
    re = integrate.dblquad(lambda ph, t: f(t, ph, 0), 0, a, 0, 2 * np.pi, epsabs=1e-13)[0]
    im = integrate.dblquad(lambda ph, t: f(t, ph, 1), 0, a, 0, 2 * np.pi, epsabs=1e-13)[0]
    ref = k0 ** 2 * 0.25j * (re + 1j * im)
    c_off, _ = richmond_coeffs(p)
    assert abs(c_off * special.hankel1(0, k0 * rho) - ref) < 1e-8 * abs(ref)


def test_reciprocity_colocated_antennas():
    # Tx == Rx on one circle, line sources all normalised by the same |H0(k0 R)|: S must be symmetric
    w = scenes.workload("c1", nx=24, ny=24, ni=12, nr=12)
    p = from_workload(w)
    ops = Operators(p, dense_gd=True)
    chi = scenes.rasterise([scenes.Shape("ellipse", 0.2, -0.1, 0.5, 0.3, 0.4, 3.0, 0.1)], 24, 24, 2.0)
    _, _, S = forward_solve(ops, chi)
    assert np.linalg.norm(S - S.T) / np.linalg.norm(S) < 1e-12


def test_dense_equals_fft_rectangular():
    p = Problem(nx=12, ny=9, side_x=2.0, side_y=1.5, k0=2 * np.pi, tx=np.array([[5.0, 0.0]]),
                rx=np.array([[0.0, 5.0]]), kx=3, ky=3)
    G = gd_dense(p)
    rng = np.random.default_rng(0)
    J = rng.standard_normal((2, 9, 12)) + 1j * rng.standard_normal((2, 9, 12))
    dense = (J.reshape(2, -1) @ G.T).reshape(J.shape)
    assert np.abs(dense - gd_apply(p, J)).max() < 1e-12 * np.abs(dense).max()
    dense_h = (J.reshape(2, -1) @ G.conj()).reshape(J.shape)          # G^H = conj(G)^T, G symmetric
    assert np.abs(dense_h - gd_apply(p, J, adjoint=True)).max() < 1e-12 * np.abs(dense_h).max()
    assert np.abs(G - G.T).max() == 0.0


def test_operator_adjoint_identities():
    p, ops = _disk_problem(16, dense=False)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((p.ni, 16, 16)) + 1j * rng.standard_normal((p.ni, 16, 16))
    y = rng.standard_normal((p.ni, 16, 16)) + 1j * rng.standard_normal((p.ni, 16, 16))
    lhs = np.vdot(y, ops.gd(x))
    rhs = np.vdot(ops.gd(y, adjoint=True), x)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    d = rng.standard_normal((p.ni, p.nr)) + 1j * rng.standard_normal((p.ni, p.nr))
    assert abs(np.vdot(d, ops.gs(x)) - np.vdot(ops.gsh(d), x)) < 1e-13 * abs(np.vdot(d, ops.gs(x)))


def test_born_limit():
    p, ops = _disk_problem(16)
    chi = 1e-4 * scenes.rasterise([scenes.Shape("disk", 0.1, 0.2, 0.5)], 16, 16, 2.0) / 1.0
    _, _, esca = forward_solve(ops, chi)
    born = (chi[None] * ops.Einc).reshape(p.ni, -1) @ ops.GS.T
    assert np.linalg.norm(esca - born) / np.linalg.norm(born) < 1e-3


def test_iterative_matches_dense():
    p, ops = _disk_problem(32, dense=True)
    chi = scenes.make_scene(scenes.workload("c2", nx=32, ny=32), 0)
    J1, _, e1 = forward_solve(ops, chi, dense_max=4096)
    J2, _, e2 = forward_solve(Operators(p), chi, dense_max=0)
    assert np.linalg.norm(e1 - e2) / np.linalg.norm(e1) < 1e-8


@pytest.mark.parametrize("eps_r", [1.5, 2.0, 3.5, 5.0])
@pytest.mark.parametrize("k0a", [0.3, 1.5, 4.0])
def test_mie_partial_waves_conserve_energy(eps_r, k0a):
    # Outside the cylinder partial wave n is J_n + a_n H_n = (H_n^(2) + (1 + 2 a_n) H_n^(1)) / 2:
    # incoming amplitude 1/2, outgoing (1 + 2 a_n) / 2.  A lossless cylinder returns all incoming
    # power, so |S_n| = |1 + 2 a_n| = 1 for every n.  This checks the matching algebra
    # independently (a sign error in a_n breaks it).  It cannot see a conjugated a_n (H^(2) for
    # H^(1), the other time convention), which the absorption test below catches.
    from oracle.mie import mie_coeffs
    k0 = 2 * np.pi
    an = mie_coeffs(k0, k0a / k0, eps_r, 30)
    assert np.abs(np.abs(1 + 2 * an) - 1).max() < 1e-10


def test_mie_lossy_cylinder_absorbs():
    # With the e^{-i w t} convention a medium with Im eps_r > 0 absorbs: every |S_n| <= 1, and the
    # low orders, which carry the power into the cylinder, lose a visible part of it.
    from oracle.mie import mie_coeffs
    k0 = 2 * np.pi
    an = mie_coeffs(k0, 0.4, 2.5 * (1 + 0.3j), 30)
    s = np.abs(1 + 2 * an)
    assert s.max() <= 1 + 1e-12
    assert s[30] < 0.99 and s[31] < 0.99 and s[29] < 0.99            # n = 0, +1, -1


def test_grid_geometry():
    # Sec. 2: an M1 x M2 uniform grid over a DOI centred on the origin.  Cell centres are
    # symmetric about 0 with spacing side / n and half a cell clear of the edges; the Richmond
    # disk has the cell's area; the scene rasteriser samples the same centres.
    p = Problem(nx=24, ny=20, side_x=2.0, side_y=1.5, k0=2 * np.pi, tx=np.zeros((1, 2)), rx=np.zeros((1, 2)),
                kx=5, ky=5)
    X, Y = p.centres()
    assert X.shape == (20, 24) and Y.shape == (20, 24)
    assert np.allclose(X[0], -X[0, ::-1]) and np.allclose(Y[:, 0], -Y[::-1, 0])
    assert np.allclose(np.diff(X[0]), 2.0 / 24) and np.allclose(np.diff(Y[:, 0]), 1.5 / 20)
    assert np.isclose(X[0, 0], -1.0 + 1.0 / 24) and np.isclose(Y[-1, 0], 0.75 - 0.75 / 20)
    assert np.isclose(np.pi * p.a_eq ** 2, (2.0 / 24) * (1.5 / 20))
    Xs, Ys = scenes.pixel_centres(24, 20, 2.0, 1.5)
    assert np.array_equal(X, Xs) and np.array_equal(Y, Ys)

"""Pins of the CCO's adjoint (Sec. 2.4, Eq. 10, 11) and of the loss with the CCO inside it.

The adjoint is pinned from outside its own code: the box mean's adjoint against the transpose of
the box matrix assembled column by column from unit images; central differences of the filter, of
the whole CCO and of the composite loss; the eps -> inf limit of the filter (linear: the double box
mean, whose adjoint is that matrix's transpose squared) and the eps -> 0 limit (the identity).
"""
import numpy as np
import pytest

import scenes
from oracle import cco, loss
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import from_workload


def box_matrix(ny, nx, r):
    """The box mean as a dense matrix, one column per unit image."""
    B = np.zeros((ny * nx, ny * nx))
    for k in range(ny * nx):
        e = np.zeros(ny * nx)
        e[k] = 1.0
        B[:, k] = cco.box_mean(e.reshape(ny, nx), r).ravel()
    return B


@pytest.mark.parametrize("shape,r", [((6, 7), 2), ((9, 5), 1), ((4, 4), 3)])
def test_box_adjoint_is_the_transpose(shape, r):
    B = box_matrix(*shape, r)
    c = np.random.default_rng(0).standard_normal(shape)
    assert np.abs(cco.box_mean_adjoint(c, r).ravel() - B.T @ c.ravel()).max() < 1e-14


def _fd(f, x, d, h):
    return (f(x + h * d) - f(x - h * d)) / (2 * h)


def test_guided_filter_adjoint_central_differences():
    rng = np.random.default_rng(1)
    I = rng.standard_normal((8, 9))
    c = rng.standard_normal(I.shape)
    for _ in range(3):
        d = rng.standard_normal(I.shape)
        fd = _fd(lambda z: np.sum(c * cco.guided_self(z, 2, 0.3)), I, d, 1e-5)
        an = np.sum(cco.guided_self_vjp(I, c, 2, 0.3) * d)
        assert abs(fd - an) < 1e-8 * max(abs(fd), 1.0), (fd, an)


def test_guided_filter_adjoint_limits():
    rng = np.random.default_rng(2)
    I = rng.standard_normal((7, 8))
    c = rng.standard_normal(I.shape)
    B = box_matrix(7, 8, 2)
    # eps -> inf: a -> 0, b -> mu, the filter is the double box mean, its adjoint B^T B^T
    assert np.abs(cco.guided_self_vjp(I, c, 2, 1e14).ravel() - B.T @ (B.T @ c.ravel())).max() < 1e-9
    # eps -> 0: a -> 1 on windows of positive variance, b -> 0, the filter and its adjoint -> identity
    assert np.abs(cco.guided_self_vjp(I, c, 2, 1e-14) - c).max() < 1e-9


def _chi(shape, rng):
    # magnitudes on both sides of tau = 3 (where the gain's derivative is large) and near 0
    mag = rng.uniform(0.0, 5.0, shape)
    return mag * np.exp(1j * rng.uniform(-0.4, 1.2, shape))


@pytest.mark.parametrize("unsharp", [False, True])
def test_cco_adjoint_central_differences(unsharp):
    rng = np.random.default_rng(3)
    chi = _chi((9, 8), rng)
    c = rng.standard_normal(chi.shape) + 1j * rng.standard_normal(chi.shape)
    kw = dict(r=2, eps=0.05, eta_max=0.1, tau=3.0, delta=0.5, unsharp=unsharp)
    g = cco.cco_vjp(chi, c, **kw)
    for _ in range(3):
        d = rng.standard_normal(chi.shape) + 1j * rng.standard_normal(chi.shape)
        fd = _fd(lambda z: np.sum(np.real(np.conj(c) * cco.cco(z, **kw))), chi, d, 1e-6)
        an = np.sum(np.real(np.conj(g) * d))
        assert abs(fd - an) < 1e-8 * abs(fd), (fd, an)


def test_cco_adjoint_gain_term_matters():
    # the eta(|chi|) path is a visible part of the adjoint where |chi| is near tau
    rng = np.random.default_rng(4)
    chi = _chi((6, 6), rng)
    c = rng.standard_normal(chi.shape) + 1j * rng.standard_normal(chi.shape)
    full = cco.cco_vjp(chi, c)
    no_gain = cco.cco_vjp(chi, c, eta_max=0.0)
    assert np.abs(full - no_gain).max() > 1e-2 * np.abs(full).max()


def _setup(**kw):
    w = scenes.workload("c1", nx=12, ny=12, ni=3, nr=6, kx=5, ky=5)
    p = from_workload(w, **kw)
    ops = Operators(p)
    chi = scenes.rasterise([scenes.Shape("disk", 0.1, 0.0, 0.45, eps_r=3.0, tan_d=0.2)], 12, 12, 2.0)
    _, _, esca = forward_solve(ops, chi)
    return p, ops, esca


@pytest.mark.parametrize("scale", [0.3, 1.0])
def test_loss_with_cco_inside_central_differences(scale):
    # heavy regulariser weights and a gain centred on the contrast present, so that the CCO's
    # adjoint carries a large share of the gradient
    p, ops, esca = _setup(cco_in_loss=True, lam_bound=1.0, lam_tv=0.3, lam_bridge=0.5, cco_tau=0.3,
                          cco_delta=0.2)
    rng = np.random.default_rng(5)
    a = scale * (rng.standard_normal((p.ni, p.ky, p.kx)) + 1j * rng.standard_normal((p.ni, p.ky, p.kx)))
    terms, g = loss.loss_grad(ops, esca, a)
    for _ in range(3):
        d = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
        fd = _fd(lambda z: loss.loss(ops, esca, z)[0], a, d, 1e-6)
        an = np.sum(np.real(np.conj(g) * d))
        assert abs(fd - an) < 1e-7 * abs(fd), (fd, an)
    # the option changes the loss and its gradient
    p0, ops0, _ = _setup(lam_bound=1.0, lam_tv=0.3, lam_bridge=0.5, cco_tau=0.3, cco_delta=0.2)
    t0, g0 = loss.loss_grad(ops0, esca, a)
    assert abs(t0[0] - terms[0]) > 1e-6 * abs(terms[0])
    assert np.linalg.norm(g - g0) > 1e-4 * np.linalg.norm(g)
    # the physics terms are the same: the CCO reaches only the regularisers
    np.testing.assert_allclose(terms[1:3], t0[1:3], rtol=1e-13)


def test_cco_inside_the_loss_of_a_constant_contrast():
    # chi_CCO of a constant image is (1 + 2 eta) chi (the filter passes constants), so the bound
    # term of a negative constant contrast is (1 + 2 eta)^2 times the plain one
    c = -0.4 + 0.1j
    img = np.full((6, 6), c)
    eta, _ = cco.gain(np.abs(img), 0.1, 3.0, 0.5)
    out = cco.cco(img)
    assert np.abs(out - (1 + 2 * eta) * img).max() < 1e-13

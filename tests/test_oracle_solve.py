"""Pins of the oracle's initialisation, Adam, CCO and solve (Sec. 2.4, 3.1, 3.3)."""
import numpy as np
import pytest
from scipy import ndimage

import scenes
from oracle import fbe, loss, solve
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import from_workload


@pytest.fixture(scope="module")
def c1_small():
    w = scenes.workload("c1", nx=16, ny=16, ni=6, nr=12, kx=5, ky=5)
    p = from_workload(w)
    ops = Operators(p, dense_gd=True)
    chi = scenes.rasterise([scenes.Shape("disk", 0.0, 0.0, 0.4, eps_r=2.0)], 16, 16, 2.0)
    _, _, esca = forward_solve(ops, chi)
    return p, ops, chi, esca


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x0 = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    t = torch.tensor(x0, dtype=torch.complex128, requires_grad=True)
    opt_t = torch.optim.Adam([t], lr=1e-2)
    ours = solve.Adam(lr=1e-2)
    x = x0.copy()
    for k in range(20):
        g = (1.0 + k) * (rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4)))
        t.grad = torch.tensor(g)
        opt_t.step()
        x = ours.step(x, g)
    assert np.abs(t.detach().numpy() - x).max() < 1e-12


def test_bp_scale_and_contrast_least_squares(c1_small):
    p, ops, chi, esca = c1_small
    chi0, R0, Jbp = solve.bp_init(ops, esca)
    # gamma minimises ||E - gamma G_S G_S^H E||: the residual is orthogonal to G_S G_S^H E
    gh = ops.gsh(esca)
    res = esca - ops.gs(Jbp)
    assert np.abs(np.sum(res * np.conj(ops.gs(gh)), axis=1)).max() < 1e-10 * np.linalg.norm(esca) ** 2
    # chi0 is the per-pixel LS fit of J = chi E_tot: normal equations hold
    etot = ops.Einc + ops.gd(Jbp)
    ne = np.sum((Jbp - chi0[None] * etot) * np.conj(etot), axis=0)
    assert np.abs(ne).max() < 1e-12
    assert np.allclose(R0, p.beta * chi0 / (p.beta * chi0 + 1))


def test_csi_step_is_exact_line_search(c1_small):
    p, ops, chi, esca = c1_small
    _, R0, _ = solve.bp_init(ops, esca)
    a0 = solve.csi_step(ops, esca, R0)
    f0 = solve.csi_loss(ops, esca, R0, np.zeros_like(a0))
    f1 = solve.csi_loss(ops, esca, R0, a0)
    assert f1 < f0
    for s in (1 - 1e-2, 1 + 1e-2, 0.5, 2.0):
        assert solve.csi_loss(ops, esca, R0, s * a0) > f1
    # and a0 points along -grad L^CSI at 0 (check against central differences of L^CSI)
    rng = np.random.default_rng(1)
    d = rng.standard_normal(a0.shape) + 1j * rng.standard_normal(a0.shape)
    h = 1e-6
    z = np.zeros_like(a0)
    fd = (solve.csi_loss(ops, esca, R0, z + h * d) - solve.csi_loss(ops, esca, R0, z - h * d)) / (2 * h)
    t = np.linalg.norm(a0)
    g_dir = np.sum(np.real(np.conj(-a0 / t) * d))            # direction of the gradient, unit scaled
    fd2 = (solve.csi_loss(ops, esca, R0, z + h * (-a0 / t)) - solve.csi_loss(ops, esca, R0, z - h * (-a0 / t))) / (2 * h)
    assert abs(fd - g_dir * fd2) < 1e-6 * abs(fd2)


def test_box_mean_matches_library_interior():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((11, 13))
    ours = solve.box_mean(a, 2)
    lib = ndimage.uniform_filter(a, size=5, mode="constant")
    assert np.abs(ours[2:-2, 2:-2] - lib[2:-2, 2:-2]).max() < 1e-13
    # corner window is 3 x 3 in-bounds
    assert abs(ours[0, 0] - a[:3, :3].mean()) < 1e-15


def test_guided_filter_limits():
    rng = np.random.default_rng(3)
    img = rng.standard_normal((12, 12))
    assert np.abs(solve.guided_self(np.full((6, 7), 2.5), 2, 1e-2) - 2.5).max() < 1e-12
    assert np.abs(solve.guided_self(img, 2, 1e-14) - img).max() < 1e-9            # eps -> 0: identity
    bb = solve.box_mean(solve.box_mean(img, 2), 2)
    assert np.abs(solve.guided_self(img, 2, 1e14) - bb).max() < 1e-9              # eps -> inf: double box


def test_cco_gain():
    # constant image at |chi| = tau: eta = eta_max / 2 and G passes constants -> (1 + 2 eta) chi (Eq. 10, 11)
    c = 3.0 + 0j
    out = solve.cco(np.full((8, 8), c))
    assert np.abs(out - (1 + 2 * 0.05) * c).max() < 1e-12
    low = solve.cco(np.full((8, 8), 0.5 + 0.5j))
    eta = 0.1 / (1 + np.exp(-(abs(0.5 + 0.5j) - 3) / 0.5))
    assert np.abs(low - (1 + 2 * eta) * (0.5 + 0.5j)).max() < 1e-12


def test_small_solve_reduces_loss_and_error(c1_small):
    p, ops, chi, esca = c1_small
    out = solve.pdf_solve(ops, esca, 60, lr=3e-2, chi_true=chi, history=True)
    L = out["losses"][:, 0]
    assert L[-1] < 0.7 * L[0]
    chi_init = loss.forward(ops, esca, out["alpha0"]).chi
    assert out["relerr"] < solve.relerr(chi_init, chi)


def test_solve_from_the_exact_coefficients():
    # With no truncation (K = M), noise-free data and no regularisers, alpha = F_T(J_true) makes
    # both residuals vanish (Eq. 6, 15, 16): the gradient is at rounding level, so the first Adam
    # step, lr g / (|g| + eps) per real component, moves alpha by at most lr max|g| / eps, and
    # chi-hat read back from the solve's final alpha is the true contrast.  (Later steps do not
    # stay put: once |g| exceeds eps, Adam's normalised step is ~lr whatever the gradient's size,
    # so the exact minimiser is not a fixed point of the loop beyond the first step.)
    w = scenes.workload("c1", nx=12, ny=12, ni=4, nr=8, kx=12, ky=12)
    p = from_workload(w, lam_bound=0.0, lam_tv=0.0, lam_bridge=0.0)
    ops = Operators(p, dense_gd=True)
    chi = scenes.rasterise([scenes.Shape("disk", 0.1, -0.05, 0.45, eps_r=2.5, tan_d=0.2)], 12, 12, 2.0)
    J, _, esca = forward_solve(ops, chi)
    a_star = fbe.analysis(J, 12, 12)
    terms, g = loss.loss_grad(ops, esca, a_star)
    gmax = max(np.abs(g.real).max(), np.abs(g.imag).max())
    assert terms[0] < 1e-24 and gmax < 1e-10
    out = solve.pdf_solve(ops, esca, 1, alpha0=a_star, chi_true=chi, apply_cco=False)
    step = out["alpha"] - a_star
    ulp = np.spacing(np.abs(a_star).max())                 # rounding of alpha + step
    assert max(np.abs(step.real).max(), np.abs(step.imag).max()) <= 1e-2 * gmax / 1e-8 + 2 * ulp
    assert out["relerr"] < 1e-6


def test_first_adam_step_descends_by_the_l1_norm(c1_small):
    # At t = 1 Adam moves each real component by -lr g / (|g| + eps), so for small lr
    # L(alpha_1) = L(alpha_0) - lr ||g||_1 + O(lr^2), with ||g||_1 summed over Re and Im parts in
    # the gradient convention g = dL/dRe + i dL/dIm.  A conjugated gradient (the sign of the
    # imaginary part flipped) or a wrong sign in the update breaks the first-order term.
    p, ops, chi, esca = c1_small
    _, R0, _ = solve.bp_init(ops, esca)
    a0 = solve.csi_step(ops, esca, R0)
    _, g = loss.loss_grad(ops, esca, a0)
    l1 = np.abs(g.real).sum() + np.abs(g.imag).sum()
    for lr in (1e-5, 1e-6):
        out = solve.pdf_solve(ops, esca, 2, lr=lr, alpha0=a0, apply_cco=False, history=True)
        L0, L1 = out["losses"][0, 0], out["losses"][1, 0]
        assert abs((L0 - L1) / lr - l1) < 2e-2 * l1, (lr, (L0 - L1) / lr, l1)

"""Pins of the oracle's coefficient-correcting network and its solve (Sec. 3, network
architecture and training settings; oracle/fcnn.py).

Central finite differences of L(alpha_(0) + Delta alpha(theta)) in the weights, the zero output
layer (first iterate = alpha_(0), first loss = the plain loss there), Adam's first step
(-lr g / (|g| + eps) on every weight), and the flat parameter layout.
"""
import numpy as np

import scenes
from oracle import fcnn, loss
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import from_workload

H = 6


def _setup(n=16, ni=4, nr=8, k=5):
    w = scenes.workload("c1", nx=n, ny=n, ni=ni, nr=nr, kx=k, ky=k)
    p = from_workload(w)
    ops = Operators(p, dense_gd=False)
    chi = scenes.rasterise([scenes.Shape("disk", 0.1, 0.0, 0.45, eps_r=2.5, tan_d=0.2)], n, n, 2.0)
    _, _, esca = forward_solve(ops, chi)
    rng = np.random.default_rng(11)
    a0 = 0.2 * (rng.standard_normal((ni, k, k)) + 1j * rng.standard_normal((ni, k, k)))
    return p, ops, chi, esca, a0


def _theta_live(k, seed=3):
    """Initial weights with a non-zero output layer, so every layer gets a gradient."""
    D = 2 * k * k
    th = scenes.fcnn_params(k, k, H, seed).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = fcnn.unpack(th, D, H)
    rng = np.random.default_rng(seed + 100)
    W3[...] = rng.uniform(-0.3, 0.3, W3.shape)
    b3[...] = rng.uniform(-0.1, 0.1, b3.shape)
    return th


def test_layout_and_zero_output_layer():
    k = 5
    D = 2 * k * k
    th = scenes.fcnn_params(k, k, H, 0)
    assert th.dtype == np.float32 and th.size == H * D + H + H * H + H + D * H + D
    W1, b1, W2, b2, W3, b3 = fcnn.unpack(th.astype(np.float64), D, H)
    assert np.all(np.abs(W1) <= 1 / np.sqrt(D)) and np.all(np.abs(W2) <= 1 / np.sqrt(H))
    assert not W3.any() and not b3.any()


def test_first_iterate_is_alpha0_and_loss_matches_plain():
    p, ops, chi, esca, a0 = _setup()
    th = scenes.fcnn_params(5, 5, H, 0).astype(np.float64)
    a, _, _ = fcnn.alpha_of(th, a0, H)
    assert np.array_equal(a, a0)
    terms, _ = fcnn.loss_grad_theta(ops, esca, a0, th, H)
    assert np.allclose(terms, loss.loss(ops, esca, a0), rtol=0, atol=0)


def test_weight_gradient_central_differences():
    p, ops, chi, esca, a0 = _setup()
    th = _theta_live(5)
    _, g = fcnn.loss_grad_theta(ops, esca, a0, th, H)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal(th.shape)
        lp = fcnn.loss_grad_theta(ops, esca, a0, th + h * d, H)[0][0]
        lm = fcnn.loss_grad_theta(ops, esca, a0, th - h * d, H)[0][0]
        fd = (lp - lm) / (2 * h)
        an = float(g @ d)
        assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3)


def test_weight_gradient_single_coordinates():
    # one weight of each layer: checks the layer order and the transposes, not just consistency
    p, ops, chi, esca, a0 = _setup()
    k, D = 5, 50
    th = _theta_live(k, seed=8)
    _, g = fcnn.loss_grad_theta(ops, esca, a0, th, H)
    offs = np.cumsum([0, H * D, H, H * H, H, D * H, D])
    h = 1e-6
    for layer in range(6):
        i = offs[layer] + (offs[layer + 1] - offs[layer]) // 3
        e = np.zeros_like(th)
        e[i] = 1.0
        fd = (fcnn.loss_grad_theta(ops, esca, a0, th + h * e, H)[0][0]
              - fcnn.loss_grad_theta(ops, esca, a0, th - h * e, H)[0][0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(np.abs(g).max(), 1e-3), layer


def test_adam_first_step_is_minus_lr_sign():
    p, ops, chi, esca, a0 = _setup()
    th = scenes.fcnn_params(5, 5, H, 1).astype(np.float64)
    _, g = fcnn.loss_grad_theta(ops, esca, a0, th, H)
    lr = 1e-2
    th1 = fcnn.AdamReal(lr=lr).step(th, g)
    # first step: m-hat = g, sqrt(v-hat) = |g|, so the move is -lr g / (|g| + eps)
    assert np.allclose(th1 - th, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    big = np.abs(g) > 1e-4
    assert np.allclose((th1 - th)[big], -lr * np.sign(g[big]), rtol=1e-4, atol=0)
    # with a zero output layer only the output layer moves on the first step
    D = 50
    n_hidden = H * D + H + H * H + H
    assert not g[:n_hidden].any() and g[n_hidden:].any()


def test_reparam_solve_lowers_the_loss():
    p, ops, chi, esca, a0 = _setup()
    th = scenes.fcnn_params(5, 5, H, 2)
    out = fcnn.reparam_solve(ops, esca, 30, th, H, lr=1e-2, alpha0=a0, chi_true=chi, history=True)
    L = out["losses"][:, 0]
    assert L[-1] < 0.5 * L[0]


def test_identity_network_closed_form():
    # H = D, W1 = W2 = W3 = I and zero biases: the network passes the positive part of its input,
    # y = ReLU(s x), so Delta alpha = (max(Re alpha_0, 0) + i max(Im alpha_0, 0)) s / s: the input
    # scale, the (Re, Im) packing, the ReLUs and the layer layout of the flat vector, all by hand.
    k = 3
    D = 2 * k * k
    eye = np.eye(D)
    th = np.concatenate([eye.ravel(), np.zeros(D), eye.ravel(), np.zeros(D), eye.ravel(), np.zeros(D)])
    rng = np.random.default_rng(3)
    a0 = rng.standard_normal((2, k, k)) + 1j * rng.standard_normal((2, k, k))
    a, _, s = fcnn.alpha_of(th, a0, D)
    ref = a0 + np.maximum(a0.real, 0) + 1j * np.maximum(a0.imag, 0)
    assert np.abs(a - ref).max() < 1e-14
    X = np.concatenate([a0.real.reshape(2, -1), a0.imag.reshape(2, -1)], axis=1)
    assert abs(s * np.sqrt(np.mean(X ** 2)) - 1.0) < 1e-14

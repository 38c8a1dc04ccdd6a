"""FP64 reference of the coefficient-correcting network and the solve built on it (test
infrastructure only: used by tests/, __graft_entry__.smoke() and bench.py's baseline leg).

The solver of Sec. 3 (network architecture) optimises the weights of a fully connected network
whose input is the initial Fourier coefficients alpha_(0) as two channels (real, imaginary parts)
and whose output is a corrective update: alpha-hat = alpha_(0) + Delta alpha; Adam with learning
rate 1e-2 acts on the weights (training settings).  The paper does not print the architecture;
the reading taken here:
  * one network shared by all incidences, applied to each incidence's K_y x K_x coefficients:
    input x_p = s [Re alpha_(0),p, Im alpha_(0),p] (D = 2 K_y K_x reals), s = 1 / RMS of alpha_(0)'s
    real components over all incidences;
  * two hidden layers of width H with ReLU, a linear output of D reals y_p;
    Delta alpha_p = (y_p[:K^2] + i y_p[K^2:]) / s;
  * hidden weights and biases uniform in +-1/sqrt(fan_in), output layer zero (the first iterate
    is alpha_(0)); flat parameter order W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [D][H], b3 [D].
The chain rule to the weights takes g = dL/dRe alpha + i dL/dIm alpha (the gradient returned by
loss.loss_grad) as dL/dy_p = [Re g_p, Im g_p] / s, then the textbook backward of the layers.

Pinned by: central finite differences of L(alpha_(0) + Delta alpha(theta)) in theta, the zero
output layer (first iterate and first loss equal the plain solve's), and Adam's first step
(every weight moves by -lr g / (|g| + eps)).
"""
from __future__ import annotations

import numpy as np

from .loss import forward, loss_grad
from .solve import bp_init, cco, csi_step, relerr


def unpack(theta: np.ndarray, D: int, H: int):
    """Views (W1, b1, W2, b2, W3, b3) of the flat parameter vector."""
    sizes = [(H, D), (H,), (H, H), (H,), (D, H), (D,)]
    out, o = [], 0
    for s in sizes:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    assert o == theta.size
    return out


def inputs(alpha0: np.ndarray):
    """Network input X [ni][D] and the scale s."""
    ni = alpha0.shape[0]
    X = np.concatenate([alpha0.real.reshape(ni, -1), alpha0.imag.reshape(ni, -1)], axis=1)
    s = 1.0 / np.sqrt(np.mean(X ** 2))
    return s * X, s


def net_forward(theta, X, H):
    """y [ni][D] and the cache for the backward pass."""
    D = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(theta, D, H)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def net_backward(theta, cache, dY, H):
    """Flat gradient of sum(dY * y) with respect to theta."""
    X, z1, h1, z2, h2 = cache
    D = X.shape[1]
    W1, b1, W2, b2, W3, b3 = unpack(theta, D, H)
    dW3 = dY.T @ h2
    db3 = dY.sum(axis=0)
    dz2 = (dY @ W3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def alpha_of(theta, alpha0, H):
    """alpha-hat = alpha_(0) + Delta alpha(theta), with the cache and scale for the backward pass."""
    ni, ky, kx = alpha0.shape
    X, s = inputs(alpha0)
    y, cache = net_forward(theta, X, H)
    k2 = ky * kx
    da = (y[:, :k2] + 1j * y[:, k2:]).reshape(ni, ky, kx) / s
    return alpha0 + da, cache, s


def loss_grad_theta(ops, esca, alpha0, theta, H):
    """Loss terms at alpha-hat(theta) and dL/dtheta."""
    a, cache, s = alpha_of(theta, alpha0, H)
    terms, g = loss_grad(ops, esca, a)
    ni = alpha0.shape[0]
    dY = np.concatenate([g.real.reshape(ni, -1), g.imag.reshape(ni, -1)], axis=1) / s
    return terms, net_backward(theta, cache, dY, H)


class AdamReal:
    """torch.optim.Adam (no weight decay, no amsgrad) on a real vector."""

    def __init__(self, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps, self.t = lr, b1, b2, eps, 0
        self.m = self.v = None

    def step(self, x, g):
        if self.m is None:
            self.m, self.v = np.zeros_like(x), np.zeros_like(x)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return x - self.lr * mh / (np.sqrt(vh) + self.eps)


def reparam_solve(ops, esca, iters, theta0, H, lr=1e-2, alpha0=None, chi_true=None, apply_cco=True,
                  history=False):
    """Whole reconstruction with the network: init (BP + CSI step unless alpha0 is given), Adam on
    theta for `iters` steps, final chi-hat at alpha-hat(theta), CCO."""
    if alpha0 is None:
        _, R0, _ = bp_init(ops, esca)
        alpha0 = csi_step(ops, esca, R0)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    opt = AdamReal(lr=lr)
    losses = []
    for _ in range(iters):
        terms, g = loss_grad_theta(ops, esca, alpha0, theta, H)
        if history:
            losses.append(terms)
        theta = opt.step(theta, g)
    alpha = alpha_of(theta, alpha0, H)[0]
    chi = forward(ops, esca, alpha).chi
    out = dict(alpha=alpha, alpha0=alpha0, theta=theta, chi=chi, losses=np.array(losses))
    out["chi_cco"] = cco(chi) if apply_cco else chi
    if chi_true is not None:
        out["relerr"] = relerr(chi, chi_true)
        out["relerr_cco"] = relerr(out["chi_cco"], chi_true)
    return out

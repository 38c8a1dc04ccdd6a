"""Learned warm start for the PDF solve (not in the paper): data, training and inference.

The network maps the measured field of one scene to initial Fourier coefficients:
  input   x = [Re, Im] of E_sca / (||E_sca||_F / sqrt(ni nr)), flattened over [ni][nr] (2 ni nr reals)
  output  y = [Re, Im] interleaved of (alpha_chi, alpha_J) with alpha_chi = F_T(chi_true) and
          alpha_J[p] = F_T(J_true[p]) truncated to the retained K x K modes (Eq. 9), i.e.
          (1 + ni) K^2 complex values.
The alpha_J part becomes alpha_(0) of the solve (pdf_solve init mode 3, which keeps the BP + CSI
start of Sec. 3.1 whenever the warm start's loss is worse); alpha_chi is an auxiliary target.

Every numerical step runs in libpdf.so: training scenes are synthesised with the library's
forward solver (pdf_forward), targets with its Fourier analysis (PDF_OP_ANA), and the network is
trained and evaluated by its BF16 tensor-core kernels (pdf_mlp_*).  This module moves arrays.
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, replace

import numpy as np

import scenes
from . import pdf


def _dev_ptr(t):
    return t.data_ptr()


class WarmStartMLP:
    """A pdf_mlp handle: linear layers of `sizes`, ReLU between hidden layers."""

    def __init__(self, sizes, batch_max, seed=0):
        import torch
        self.sizes = list(sizes)
        self.nl = len(sizes) - 1
        lib = pdf.load()
        arr = (ctypes.c_int32 * len(sizes))(*sizes)
        h = ctypes.c_void_p()
        pdf._check(lib.pdf_mlp_create(self.nl, arr, batch_max, ctypes.byref(h)))
        self.h = h.value
        self.batch_max = batch_max
        self.loss_dev = torch.zeros(8, dtype=torch.float64, device="cuda")
        rng = np.random.default_rng(seed)
        for l in range(self.nl):
            fan_in = sizes[l]
            bound = math.sqrt(6.0 / fan_in) if l + 1 < self.nl else math.sqrt(1.0 / fan_in)
            W = rng.uniform(-bound, bound, size=(sizes[l + 1], fan_in)).astype(np.float32)
            b = np.zeros(sizes[l + 1], np.float32)
            self.set_params(l, W, b)

    def set_params(self, l, W, b):
        W = np.ascontiguousarray(W, np.float32)
        b = np.ascontiguousarray(b, np.float32)
        pdf._check(pdf.load().pdf_mlp_set_params(self.h, l, W.ctypes.data, b.ctypes.data, pdf._stream(None)))

    def get_params(self, l):
        o, i = self.sizes[l + 1], self.sizes[l]
        W = np.empty((o, i), np.float32)
        b = np.empty(o, np.float32)
        dW = np.empty((o, i), np.float32)
        db = np.empty(o, np.float32)
        pdf._check(pdf.load().pdf_mlp_get_params(self.h, l, W.ctypes.data, b.ctypes.data, dW.ctypes.data,
                                                 db.ctypes.data, pdf._stream(None)))
        return W, b, dW, db

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], self.sizes[-1]), dtype=torch.float32, device="cuda")
        pdf._check(pdf.load().pdf_mlp_forward(self.h, _dev_ptr(X), _dev_ptr(Y), X.shape[0], pdf._stream(None)))
        return Y

    def loss_grad(self, X, T):
        pdf._check(pdf.load().pdf_mlp_loss_grad(self.h, _dev_ptr(X), _dev_ptr(T), X.shape[0],
                                                _dev_ptr(self.loss_dev), pdf._stream(None)))
        return self.loss_dev[0]

    def train_step(self, X, T, lr):
        pdf._check(pdf.load().pdf_mlp_train_step(self.h, _dev_ptr(X), _dev_ptr(T), X.shape[0], float(lr),
                                                 _dev_ptr(self.loss_dev), pdf._stream(None)))
        return self.loss_dev[0]

    def close(self):
        if getattr(self, "h", None):
            pdf.load().pdf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(esca):
    """x from E_sca [B][ni][nr] complex64 (device): each scene divided by its RMS magnitude, [Re, Im]
    interleaved, flattened (pdf_mlp_features)."""
    import torch
    esca = esca.contiguous()
    B = esca.shape[0]
    n = esca[0].numel()
    X = torch.empty((B, 2 * n), dtype=torch.float32, device=esca.device)
    pdf._check(pdf.load().pdf_mlp_features(_dev_ptr(esca), B, n, _dev_ptr(X), pdf._stream(None)))
    return X


@dataclass
class Dataset:
    X: object           # [n][2 ni nr] float32 device
    T: object           # [n][2 (1 + ni) K^2] float32 device
    chi: object         # [n][ny][nx] complex64 device (ground truth)
    esca: object        # [n][ni][nr] complex64 device (noisy measured data)
    seconds: float


def generate(prob: "pdf.Problem", w, n: int, seed0: int, noise=(0.05, 0.10), tol=1e-5) -> Dataset:
    """n scenes of workload w (its scene recipe), synthesised with the library's forward solver."""
    import torch
    t0 = time.perf_counter()
    K2 = w.kx * w.ky
    X = torch.empty((n, 2 * w.ni * w.nr), dtype=torch.float32, device="cuda")
    T = torch.empty((n, 2 * (1 + w.ni) * K2), dtype=torch.float32, device="cuda")
    CH = torch.empty((n, w.ny, w.nx), dtype=torch.complex64, device="cuda")
    ES = torch.empty((n, w.ni, w.nr), dtype=torch.complex64, device="cuda")
    chis = []
    for s in range(n):
        seed = seed0 + s
        chi = scenes.make_scene(w, seed)
        chi_d = torch.from_numpy(chi.astype(np.complex64)).cuda()
        CH[s] = chi_d
        esca, J, _ = prob.forward(chi_d, tol=tol, max_iter=3000)
        rng = np.random.default_rng(10_000_000 + seed)
        nu = float(rng.uniform(*noise))
        noisy = scenes.add_awgn(esca.cpu().numpy().astype(np.complex128), nu, rng).astype(np.complex64)
        ES[s] = torch.from_numpy(noisy).cuda()
        aJ = prob.op(pdf.OP_ANA, J)                                      # [ni][ky][kx]
        tgt = torch.empty((1 + w.ni, w.ky, w.kx), dtype=torch.complex64, device="cuda")
        tgt[1:] = aJ
        T[s] = torch.view_as_real(tgt).reshape(-1)
        chis.append(chi_d)
    # alpha_chi: F_T of chi, ni scenes per analysis call (the operator is batched over planes)
    for g0 in range(0, n, w.ni):
        g = chis[g0:g0 + w.ni]
        planes = torch.zeros((w.ni, w.ny, w.nx), dtype=torch.complex64, device="cuda")
        for k, c in enumerate(g):
            planes[k] = c
        ac = prob.op(pdf.OP_ANA, planes)
        for k in range(len(g)):
            T[g0 + k, : 2 * K2] = torch.view_as_real(ac[k].contiguous()).reshape(-1)
    X[:] = features(ES)
    torch.cuda.synchronize()
    return Dataset(X, T, CH, ES, time.perf_counter() - t0)


def train(net: WarmStartMLP, data: Dataset, steps: int, batch: int, lr=1e-3, seed=0, log_every=0):
    """Adam on random mini-batches; cosine-decayed learning rate.  Returns the loss history."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    n = data.X.shape[0]
    hist = []
    for k in range(steps):
        idx = torch.randint(0, n, (batch,), device="cuda", generator=g)
        lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
        loss = net.train_step(data.X[idx].contiguous(), data.T[idx].contiguous(), lr_k)
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append((k, float(loss)))
    torch.cuda.synchronize()
    return hist


def predict_alpha(net: WarmStartMLP, esca, w):
    """alpha_(0) [ni][ky][kx] complex64 for one scene's measured field [ni][nr] (device)."""
    import torch
    y = net.forward(features(esca[None]))
    c = torch.view_as_complex(y.reshape(-1, 2).contiguous()).reshape(1 + w.ni, w.ky, w.kx)
    return c[1:].contiguous()


def evaluate(prob, net, data: Dataset, w, iters: int, every: int = 5):
    """Per scene: plain solve (BP + CSI) and warm-started solve, with RelErr histories.

    Returns a list of dicts: relerr_plain (final, after CCO), iterations the warm start needs to
    reach it (None if never), whether the warm start was kept, and both loss values at start."""
    import torch
    out = []
    for s in range(data.X.shape[0]):
        prob.set_data(data.esca[s].contiguous())
        chi_t = data.chi[s].contiguous()
        plain = prob.solve(iters=iters, chi_true=chi_t, history_every=every)
        a0 = predict_alpha(net, data.esca[s], w)
        warm = prob.solve(iters=iters, init=3, alpha0=a0, chi_true=chi_t, history_every=every)
        hp = plain["history"].cpu().numpy()
        hw = warm["history"].cpu().numpy()
        target = plain["relerr_cco"]
        reach = None
        for r in range(hw.shape[0]):
            if hw[r, 7] <= target:
                reach = r * every
                break
        out.append(dict(relerr_plain=target, relerr_warm=warm["relerr_cco"], iters_to_plain=reach,
                        used_warm=warm["used_warm_start"], loss0_plain=hp[0, 0], loss0_warm=hw[0, 0],
                        relerr0_plain=hp[0, 7], relerr0_warm=hw[0, 7]))
    return out

"""Shared set-up of the GPU parity tests: one geometry on both sides (oracle and CUDA library)."""
import numpy as np

import scenes
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import from_workload

# FP32 path tolerance against the FP64 oracle, norm-wise relative (loss, gradient, operators).
TOL_FP32 = 1e-5


def rel(a, b):
    """Norm-wise relative error ||a - b|| / ||b||."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """Element-wise error max |a - b| / max |b|: a wrong small block (a few modes, the edge pixels)
    that a norm-wise ratio can hide under a large correct one shows up here."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def assert_close(name, gpu, ref, tol, tol_elem=None):
    """Both the norm-wise and the element-wise error of `gpu` against the oracle's `ref` within
    tol (tol_elem for the element-wise one when given)."""
    gpu = gpu.cpu().numpy() if hasattr(gpu, "cpu") else np.asarray(gpu)
    e, m = rel(gpu, ref), maxrel(gpu, ref)
    te = tol if tol_elem is None else tol_elem
    print(f"{name}: norm-wise {e:.2e}, element-wise {m:.2e}")
    assert e < tol, f"{name}: norm-wise rel err {e:.2e} >= {tol:g}"
    assert m < te, f"{name}: element-wise err {m:.2e} >= {te:g} (norm-wise {e:.2e})"


class Case:
    """A workload instantiated for both sides with identical complex64-rounded measured data."""

    def __init__(self, w, seed=0, noise=None):
        self.w = w
        self.p = from_workload(w)
        self.ops = Operators(self.p)
        self.chi = scenes.make_scene(w, seed)
        _, _, esca = forward_solve(self.ops, self.chi)
        nu = w.noise if noise is None else noise
        esca = scenes.add_awgn(esca, nu, np.random.default_rng(1000 + seed))
        self.esca32 = esca.astype(np.complex64)
        self.esca = self.esca32.astype(np.complex128)       # the oracle sees exactly the GPU's data

    def problem(self, **kw):
        from paper_2602_13805_gb300 import pdf
        return pdf.Problem.from_workload(self.w, esca=self.esca32, **kw)

    def alpha(self, scale=0.3, seed=0):
        rng = np.random.default_rng(seed)
        return scenes.random_coeffs(self.p.ni, self.p.ky, self.p.kx, scale, rng).astype(np.complex64)


# geometries spanning several tiles and ragged tails: (name, overrides)
SMALL_CASES = [
    ("g16", dict(nx=16, ny=16, ni=4, nr=8, kx=5, ky=5)),
    ("g24x20", dict(nx=24, ny=20, ni=5, nr=7, kx=7, ky=5)),          # padded lengths 48 = 2^4 3, ragged row tiles
    ("c1", dict()),
]

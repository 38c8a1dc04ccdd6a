"""Shared set-up of the GPU parity tests: one geometry on both sides (oracle and CUDA library)."""
import numpy as np

import scenes
from oracle.forward import forward_solve
from oracle.green import Operators
from oracle.problem import from_workload

# FP32 path tolerance against the FP64 oracle, norm-wise relative (loss, gradient, operators).
TOL_FP32 = 1e-5


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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

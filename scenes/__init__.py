"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds input generation only: measurement geometry (antennas on a
circle), rasterised contrast maps (disks, ellipses, rings), additive white
Gaussian noise, and the named workload presets.  It contains none of the
method's arithmetic (no Green's functions, no loss, no solver), so both sides
can draw identical inputs from it without sharing any of the computation.

Units: lengths in free-space wavelengths (lambda = 1), so k0 = 2*pi.  The domain
of interest (DOI) is centred on the origin; arrays are row-major [y][x] with x
fastest.  Contrast chi = eps_r * (1 + i tan_delta) - 1 (time factor e^{-i w t}),
which gives Re chi >= 0 and Im chi >= 0 for physical media (Sec. 2.2, Eq. 7).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass
class Workload:
    """One synthetic inverse-scattering workload (geometry + scene recipe)."""
    name: str
    nx: int                     # M1, pixels along x
    ny: int                     # M2, pixels along y
    side: float                 # DOI side length in wavelengths (square DOI)
    ni: int                     # number of incidences (transmitters)
    nr: int                     # number of receivers
    radius: float               # antenna circle radius in wavelengths
    kx: int                     # Fourier truncation along x (odd: symmetric; even: corner blocks)
    ky: int
    iters: int = 300            # Adam iterations of one reconstruction
    noise: float = 0.0          # relative AWGN level nu (0.1 = "10 %")
    scene: str = "disk"         # scene recipe name, see make_scene
    beta: complex = 6.0 + 0.0j  # CIE parameter (Sec. 4.1 picks beta = 6)
    inc_kind: int = 0           # 0 = line source on the Tx circle, 1 = plane wave
    k0: float = TWO_PI

    @property
    def m(self) -> int:
        return self.nx * self.ny


# Named workloads.  Sizes follow the five synthetic configurations of the
# measurement contract; "cP" is shaped like the paper's own numerical setup
# (Sec. 4: 64x64 grid over a 2-lambda DOI, 36 Tx / 36 Rx on a 20-lambda circle,
# M_F = 7 so 2*M_F = 14 retained indices per axis, beta = 6).
WORKLOADS = {
    "c1": Workload("c1", 32, 32, 2.0, 8, 16, 5.0, 11, 11, iters=300, noise=0.0, scene="disk"),
    "c2": Workload("c2", 64, 64, 2.0, 16, 32, 5.0, 15, 15, iters=300, noise=0.10, scene="two_disks"),
    "c3": Workload("c3", 128, 128, 3.0, 36, 72, 5.0, 21, 21, iters=300, noise=0.0, scene="ellipses"),
    "c4": Workload("c4", 64, 64, 2.0, 16, 32, 5.0, 15, 15, iters=300, noise=0.075, scene="random_mix"),
    "c5": Workload("c5", 192, 192, 4.0, 64, 128, 6.0, 31, 31, iters=300, noise=0.10, scene="ring_mix"),
    "cP": Workload("cP", 64, 64, 2.0, 36, 36, 20.0, 14, 14, iters=100, noise=0.0, scene="two_disks"),
}


def workload(name: str, **overrides) -> Workload:
    return replace(WORKLOADS[name], **overrides)


# ---------------------------------------------------------------------------
# Measurement geometry
# ---------------------------------------------------------------------------

def antennas(n: int, radius: float, phase: float = 0.0) -> np.ndarray:
    """n points equally spaced on a circle, starting at angle `phase`: [n][2] float64."""
    ang = phase + TWO_PI * np.arange(n) / n
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)


def perturb_antennas(xy: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    """Gaussian position jitter of standard deviation `sigma` on each coordinate (Sec. 4.5)."""
    return xy + sigma * rng.standard_normal(xy.shape)


def pixel_centres(nx: int, ny: int, side_x: float, side_y: float) -> Tuple[np.ndarray, np.ndarray]:
    """Cell-centre coordinates of the DOI grid, X and Y as [ny][nx] float64."""
    dx, dy = side_x / nx, side_y / ny
    xs = -0.5 * side_x + (np.arange(nx) + 0.5) * dx
    ys = -0.5 * side_y + (np.arange(ny) + 0.5) * dy
    return np.meshgrid(xs, ys)


# ---------------------------------------------------------------------------
# Scene rasterisation (pixel-centre inclusion)
# ---------------------------------------------------------------------------

@dataclass
class Shape:
    kind: str                   # "disk" | "ellipse" | "ring"
    cx: float
    cy: float
    a: float                    # disk radius / ellipse semi-axis x' / ring outer radius
    b: float = 0.0              # ellipse semi-axis y' / ring inner radius
    theta: float = 0.0          # ellipse orientation
    eps_r: float = 2.0
    tan_d: float = 0.0

    @property
    def chi(self) -> complex:
        return self.eps_r * (1.0 + 1j * self.tan_d) - 1.0

    def bound_radius(self) -> float:
        return self.a if self.kind != "ellipse" else max(self.a, self.b)

    def mask(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        dx, dy = X - self.cx, Y - self.cy
        if self.kind == "disk":
            return dx * dx + dy * dy <= self.a * self.a
        if self.kind == "ring":
            r2 = dx * dx + dy * dy
            return (r2 <= self.a * self.a) & (r2 >= self.b * self.b)
        c, s = math.cos(self.theta), math.sin(self.theta)
        u, v = c * dx + s * dy, -s * dx + c * dy
        return (u / self.a) ** 2 + (v / self.b) ** 2 <= 1.0


def rasterise(shapes: List[Shape], nx: int, ny: int, side: float) -> np.ndarray:
    """Contrast map chi [ny][nx] complex128; later shapes overwrite earlier ones."""
    X, Y = pixel_centres(nx, ny, side, side)
    chi = np.zeros((ny, nx), dtype=np.complex128)
    for sh in shapes:
        chi[sh.mask(X, Y)] = sh.chi
    return chi


def _place(rng: np.random.Generator, shapes: List[Shape], new: Shape, side: float,
           margin: float = 0.05, tries: int = 200) -> Optional[Shape]:
    """Random centre so that `new` lies inside the DOI and clear of `shapes` (bounding circles)."""
    r = new.bound_radius()
    half = 0.5 * side - r - margin
    if half <= 0:
        return None
    for _ in range(tries):
        cx, cy = rng.uniform(-half, half, size=2)
        ok = all(math.hypot(cx - s.cx, cy - s.cy) > r + s.bound_radius() + margin for s in shapes)
        if ok:
            return replace(new, cx=float(cx), cy=float(cy))
    return None


def scene_shapes(w: Workload, seed: int) -> List[Shape]:
    """The shapes of one seeded scene of workload `w` (recipes of the measurement contract)."""
    rng = np.random.default_rng(seed)
    if w.scene == "disk":                       # one centred lossless disk, r = 0.4, eps_r = 2
        return [Shape("disk", 0.0, 0.0, 0.4, eps_r=2.0)]
    if w.scene == "two_disks":                  # r = 0.3, edge gap 0.05, eps_r = 3.5, lossless
        off = 0.3 + 0.025
        return [Shape("disk", -off, 0.0, 0.3, eps_r=3.5), Shape("disk", off, 0.0, 0.3, eps_r=3.5)]
    if w.scene in ("ellipses", "random_mix"):
        n = int(rng.integers(1, 4))
        out: List[Shape] = []
        for _ in range(n):
            if w.scene == "ellipses":
                eps = float(rng.uniform(2.0, 4.0))
                tand = float(rng.uniform(0.0, 0.3))
                kind = "ellipse"
            else:
                eps = float(rng.uniform(1.5, 4.0))
                tand = 0.0
                kind = "disk" if rng.uniform() < 0.5 else "ellipse"
            a = float(rng.uniform(0.2, 0.6) if w.scene == "ellipses" else rng.uniform(0.15, 0.45))
            b = float(rng.uniform(0.2, 0.6) if w.scene == "ellipses" else rng.uniform(0.15, 0.45))
            if kind == "disk":
                b = a
            sh = Shape(kind, 0.0, 0.0, a, b, float(rng.uniform(0, math.pi)), eps, tand)
            placed = _place(rng, out, sh, w.side)
            if placed is not None:
                out.append(placed)
        return out
    if w.scene == "ring_mix":                   # a high-contrast ring + two lossy scatterers
        out = []
        ring = Shape("ring", 0.0, 0.0, 0.8, 0.5, 0.0, 5.0, 0.1)
        out.append(_place(rng, out, ring, w.side))
        disk = Shape("disk", 0.0, 0.0, float(rng.uniform(0.3, 0.45)), eps_r=float(rng.uniform(2.5, 3.5)),
                     tan_d=float(rng.uniform(0.05, 0.2)))
        ell = Shape("ellipse", 0.0, 0.0, float(rng.uniform(0.3, 0.6)), float(rng.uniform(0.2, 0.4)),
                    float(rng.uniform(0, math.pi)), float(rng.uniform(2.0, 3.0)), float(rng.uniform(0.0, 0.1)))
        for sh in (disk, ell):
            p = _place(rng, out, sh, w.side)
            if p is not None:
                out.append(p)
        return out
    raise ValueError(f"unknown scene recipe {w.scene!r}")


def make_scene(w: Workload, seed: int) -> np.ndarray:
    """Seeded contrast map chi_true [ny][nx] complex128 of workload `w`."""
    return rasterise(scene_shapes(w, seed), w.nx, w.ny, w.side)


def geometry(w: Workload) -> Tuple[np.ndarray, np.ndarray]:
    """Tx and Rx positions ([ni][2], [nr][2]) on the workload's antenna circle."""
    return antennas(w.ni, w.radius), antennas(w.nr, w.radius)


# ---------------------------------------------------------------------------
# Noise and random coefficient draws
# ---------------------------------------------------------------------------

def add_awgn(esca: np.ndarray, nu: float, rng: np.random.Generator) -> np.ndarray:
    """Complex AWGN whose Frobenius norm is nu * ||esca|| in expectation (Sec. 4.2)."""
    if nu <= 0.0:
        return esca.copy()
    sig = nu * np.linalg.norm(esca) / math.sqrt(2.0 * esca.size)
    n = rng.standard_normal(esca.shape) + 1j * rng.standard_normal(esca.shape)
    return esca + sig * n


def snr_db_to_nu(snr_db: float) -> float:
    return 10.0 ** (-snr_db / 20.0)


def fcnn_params(ky: int, kx: int, hidden: int, seed: int) -> np.ndarray:
    """Initial weights of the coefficient-correcting network, float32, flat in the order
    W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [D][H], b3 [D] with D = 2 ky kx: the hidden layers
    uniform in +-1/sqrt(fan_in) (the common default for linear layers), the output layer zero so the
    first iterate is alpha_(0) itself.  Seeded input data for both implementations."""
    D, H = 2 * ky * kx, hidden
    rng = np.random.default_rng(seed)
    b_in, b_h = 1.0 / np.sqrt(D), 1.0 / np.sqrt(H)
    parts = [rng.uniform(-b_in, b_in, H * D), rng.uniform(-b_in, b_in, H),
             rng.uniform(-b_h, b_h, H * H), rng.uniform(-b_h, b_h, H),
             np.zeros(D * H), np.zeros(D)]
    return np.concatenate(parts).astype(np.float32)


def random_coeffs(ni: int, ky: int, kx: int, scale: float, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. complex Gaussian coefficient array [ni][ky][kx] complex128."""
    return scale * (rng.standard_normal((ni, ky, kx)) + 1j * rng.standard_normal((ni, ky, kx)))

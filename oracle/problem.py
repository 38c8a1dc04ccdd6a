"""Problem description shared by the oracle's modules (Sec. 2, Sec. 3.2).

The DOI is an M1 x M2 grid of square-ish pulse cells centred on the origin
(Sec. 2, "discretized into an M1 x M2 uniform grid").  Lengths are in
wavelengths when k0 = 2*pi.  Arrays over the grid are [y][x] with x fastest.

Pinned by tests/test_oracle_physics.py::test_grid_geometry: centres symmetric about the origin
with spacing side / n, half a cell clear of the edges, the equal-area Richmond radius, and the
same centres as the scene rasteriser.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    nx: int
    ny: int
    side_x: float
    side_y: float
    k0: float
    tx: np.ndarray              # [ni][2] transmitter positions (or plane-wave directions)
    rx: np.ndarray              # [nr][2] receiver positions
    kx: int                     # retained Fourier indices along x
    ky: int                     # retained Fourier indices along y
    beta: complex = 6.0         # CIE parameter, Eq. (6)-(7)
    inc_kind: int = 0           # 0 = line source, 1 = plane wave
    lam_bound: float = 1e-3     # lambda_1, Sec. 3.2
    lam_tv: float = 1e-5        # lambda_2
    lam_bridge: float = 1e-5    # lambda_3
    tau_b: float = 0.5          # bridge threshold tau_B, Eq. (19)
    eps_tv: float = 1e-8        # smoothing inside the TV square root (reading: Eq. 18 is not differentiable at 0)
    eps_abs: float = 1e-12      # smoothing inside |chi| of the bridge loss (reading of Eq. 19)
    q_min: float = 1e-6         # clamp of |1 - R| in chi = R / (beta (1 - R)) (reading of Eq. 7 near R = 1)
    # CCO of Sec. 2.4 (Eq. 10, 11): guided-filter box radius and regulariser, gain eta_max, tau, delta.
    # cco_in_loss: the regularisers of Eq. (17)-(19) act on chi_CCO instead of chi-hat (the CCO inside
    # the loss); otherwise the CCO only post-processes the solve's output.
    cco_in_loss: bool = False
    cco_radius: int = 2
    cco_eps: float = 1e-2
    cco_eta_max: float = 0.1
    cco_tau: float = 3.0
    cco_delta: float = 0.5

    @property
    def ni(self) -> int:
        return int(self.tx.shape[0])

    @property
    def nr(self) -> int:
        return int(self.rx.shape[0])

    @property
    def m(self) -> int:
        return self.nx * self.ny

    @property
    def dx(self) -> float:
        return self.side_x / self.nx

    @property
    def dy(self) -> float:
        return self.side_y / self.ny

    @property
    def a_eq(self) -> float:
        """Radius of the disk with the cell's area (Richmond's circular-cell approximation)."""
        return math.sqrt(self.dx * self.dy / math.pi)

    def centres(self):
        xs = -0.5 * self.side_x + (np.arange(self.nx) + 0.5) * self.dx
        ys = -0.5 * self.side_y + (np.arange(self.ny) + 0.5) * self.dy
        return np.meshgrid(xs, ys)


def from_workload(w, tx=None, rx=None, **kw) -> Problem:
    """Build a Problem from a scenes.Workload (antennas on the workload's circle unless given)."""
    import scenes
    if tx is None or rx is None:
        t, r = scenes.geometry(w)
        tx = t if tx is None else tx
        rx = r if rx is None else rx
    return Problem(nx=w.nx, ny=w.ny, side_x=w.side, side_y=w.side, k0=w.k0, tx=np.asarray(tx, float),
                   rx=np.asarray(rx, float), kx=w.kx, ky=w.ky, beta=complex(w.beta),
                   inc_kind=w.inc_kind, **kw)

"""Truncated Fourier basis expansion of the induced current (Sec. 2.3, Eq. 9).

J = [F_1 ... F_M0] alpha with F_k the (unitary) 2-D DFT basis functions of the
retained low-frequency modes; alpha = F_T(J) and J = F*_T(alpha).

Readings: the DFT is unitary ("ortho"), because the paper leaves the
normalisation open; per axis of length M the K retained indices are the first
ceil(K/2) non-negative frequencies and the last floor(K/2) negative ones, i.e.
storage slot j holds DFT index j for j < ceil(K/2) and M - K + j otherwise.  For
K = 2 M_F this is exactly the paper's four M_F x M_F corner blocks (M0 = 4 M_F^2);
for odd K it is the symmetric set {-(K-1)/2 .. (K-1)/2}.

Pinned by: brute-force sums of explicit basis functions, Phi^H Phi = I on the
retained set, and adjoint identities (tests/test_oracle_fbe.py).
"""
from __future__ import annotations

import numpy as np
from scipy import fft as sfft


def mode_indices(K: int, M: int) -> np.ndarray:
    if K > M or K < 1:
        raise ValueError("truncation K must be in [1, M]")
    h = (K + 1) // 2
    return np.array([j if j < h else M - K + j for j in range(K)], dtype=np.int64)


def synth(alpha: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """J = F*_T(alpha): [..., ky, kx] -> [..., ny, nx] (zero-filled spectrum, unitary inverse DFT)."""
    ky, kx = alpha.shape[-2:]
    iy, ix = mode_indices(ky, ny), mode_indices(kx, nx)
    full = np.zeros(alpha.shape[:-2] + (ny, nx), dtype=np.complex128)
    full[..., iy[:, None], ix[None, :]] = alpha
    return sfft.ifft2(full, norm="ortho")


def analysis(J: np.ndarray, ky: int, kx: int) -> np.ndarray:
    """F_T(J) restricted to the retained modes = Phi^H J: [..., ny, nx] -> [..., ky, kx]."""
    ny, nx = J.shape[-2:]
    iy, ix = mode_indices(ky, ny), mode_indices(kx, nx)
    full = sfft.fft2(J, norm="ortho")
    return full[..., iy[:, None], ix[None, :]]

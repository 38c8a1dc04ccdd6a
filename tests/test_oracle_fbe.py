"""Pins of the oracle's Fourier basis expansion (Eq. 9) against explicit basis functions."""
import numpy as np
import pytest

from oracle import fbe


def test_mode_sets():
    # odd K: symmetric set {-(K-1)/2 .. (K-1)/2}; K = 2 M_F: the paper's four corner blocks
    assert list(fbe.mode_indices(5, 16)) == [0, 1, 2, 14, 15]
    mf = 7
    assert sorted(fbe.mode_indices(2 * mf, 64)) == list(range(mf)) + list(range(64 - mf, 64))
    with pytest.raises(ValueError):
        fbe.mode_indices(17, 16)


@pytest.mark.parametrize("ny,nx,ky,kx", [(6, 8, 3, 5), (9, 7, 4, 3), (8, 8, 8, 8)])
def test_synth_is_sum_of_basis_functions(ny, nx, ky, kx):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((2, ky, kx)) + 1j * rng.standard_normal((2, ky, kx))
    fy = [j if j < (ky + 1) // 2 else j - ky for j in range(ky)]     # signed frequencies
    fx = [j if j < (kx + 1) // 2 else j - kx for j in range(kx)]
    ref = np.zeros((2, ny, nx), complex)
    for y in range(ny):
        for x in range(nx):
            for jy in range(ky):
                for jx in range(kx):
                    basis = np.exp(2j * np.pi * (fy[jy] * y / ny + fx[jx] * x / nx)) / np.sqrt(nx * ny)
                    ref[:, y, x] += a[:, jy, jx] * basis
    assert np.abs(fbe.synth(a, ny, nx) - ref).max() < 1e-12


def test_analysis_is_adjoint_and_left_inverse():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 5, 7)) + 1j * rng.standard_normal((3, 5, 7))
    J = rng.standard_normal((3, 12, 10)) + 1j * rng.standard_normal((3, 12, 10))
    assert np.abs(fbe.analysis(fbe.synth(a, 12, 10), 5, 7) - a).max() < 1e-12
    lhs = np.vdot(J, fbe.synth(a, 12, 10))
    rhs = np.vdot(fbe.analysis(J, 5, 7), a)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)

"""Host logic of the robustness studies (paper_2602_13805_gb300/studies.py): the antenna jitter of
Sec. 4.5 is reproducible per (seed, deviation, realisation), moves every antenna independently
with the requested standard deviation, and converts millimetres at 400 MHz to wavelengths."""
import numpy as np

import scenes
from paper_2602_13805_gb300 import studies


def test_wavelength_at_400_mhz():
    assert abs(studies.LAMBDA_M - 0.7494811) < 1e-6


def test_realisations_are_reproducible_and_distinct():
    w = scenes.workload("cP")
    a = studies.realisation_geometry(w, 0.004, studies.jitter_rng(0, 2, 5))
    b = studies.realisation_geometry(w, 0.004, studies.jitter_rng(0, 2, 5))
    c = studies.realisation_geometry(w, 0.004, studies.jitter_rng(0, 2, 6))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_offsets_have_the_requested_deviation():
    w = scenes.workload("cP", ni=2000, nr=2000)
    tx0, rx0 = scenes.geometry(w)
    sig = 3e-3 / studies.LAMBDA_M
    tx, rx = studies.realisation_geometry(w, sig, studies.jitter_rng(1, 0, 0))
    d = np.concatenate([(tx - tx0).ravel(), (rx - rx0).ravel()])
    assert abs(d.std() / sig - 1.0) < 0.03 and abs(d.mean()) < 0.05 * sig
    # transmitters and receivers move independently
    assert not np.allclose(tx - tx0, rx - rx0)

"""Checks of the gamma-index helper on analytic distributions."""
import numpy as np

from tests._gamma import gamma_pass_rate


def _blob(shift_mm=0.0, scale=1.0, n=24, vox=2.0, width=8.0):
    z, y, x = np.meshgrid(*(np.arange(n) * vox,) * 3, indexing="ij")
    c = n * vox / 2
    return scale * np.exp(-((x - c - shift_mm) ** 2 + (y - c) ** 2 + (z - c) ** 2) / (2 * width ** 2))


def test_identical_passes():
    a = _blob()
    assert gamma_pass_rate(a, a, (2.0, 2.0, 2.0)) == 1.0


def test_small_shift_passes_large_shift_fails():
    a = _blob()
    assert gamma_pass_rate(a, _blob(shift_mm=1.0), (2.0, 2.0, 2.0)) == 1.0
    assert gamma_pass_rate(a, _blob(shift_mm=6.0), (2.0, 2.0, 2.0)) < 0.9


def test_dose_scale():
    # a broad, nearly flat distribution: a dose scale cannot be absorbed by distance
    a = _blob(width=40.0)
    assert gamma_pass_rate(a, _blob(scale=1.01, width=40.0), (2.0, 2.0, 2.0)) == 1.0
    assert gamma_pass_rate(a, _blob(scale=1.08, width=40.0), (2.0, 2.0, 2.0)) < 0.5

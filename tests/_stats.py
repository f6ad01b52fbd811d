"""Statistical helpers shared by the tests (no transport arithmetic here)."""
from __future__ import annotations

import numpy as np
from scipy import stats


def chi2_pvalue(samples: np.ndarray, pdf, grid: np.ndarray, n_bins: int = 40) -> float:
    """Chi-square goodness of fit of ``samples`` to the density ``pdf``.

    ``grid`` is a fine, increasing grid covering the support; the CDF is built by
    trapezoidal integration on it and the bins are equal-probability quantiles
    of that CDF, which keeps every bin well populated for peaked densities.
    """
    f = np.asarray([pdf(x) for x in grid], dtype=np.float64)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(grid))])
    cdf /= cdf[-1]
    q = np.linspace(0.0, 1.0, n_bins + 1)
    edges = np.interp(q, cdf, grid)
    edges[0], edges[-1] = grid[0] - 1e-12, grid[-1] + 1e-12
    expected = np.diff(np.interp(edges, grid, cdf, left=0.0, right=1.0)) * len(samples)
    observed, _ = np.histogram(samples, bins=edges)
    keep = expected > 5
    obs, exp = observed[keep], expected[keep]
    exp = exp * obs.sum() / exp.sum()
    return float(stats.chisquare(obs, exp).pvalue)


def within_sigma(x: float, expected: float, sigma: float, k: float = 3.0) -> bool:
    return abs(x - expected) <= k * sigma


def three_sigma_pass_rate(d_a, s_a, d_b, s_b, mask) -> float:
    """Fraction of voxels in ``mask`` with |d_a - d_b| <= 3 sqrt(s_a^2 + s_b^2)."""
    diff = np.abs(d_a - d_b)[mask]
    tol = 3.0 * np.sqrt(s_a ** 2 + s_b ** 2)[mask]
    return float(np.mean(diff <= tol)) if diff.size else 1.0

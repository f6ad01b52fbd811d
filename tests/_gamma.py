"""Gamma index (Low et al.; GPUMCD §II.D) for pass-rate checks.

Global dose criterion dD = dd_frac * max(reference), distance criterion dd_mm.
The evaluated distribution is interpolated trilinearly and searched on a
lattice of spacing dd_mm / 10 within a sphere of radius dd_mm: beyond dd_mm the
distance term alone exceeds 1, so the search decides gamma <= 1 exactly up to
the lattice spacing.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import map_coordinates


def gamma_pass_rate(ref: np.ndarray, ev: np.ndarray, voxel_mm, dd_frac: float = 0.02,
                    dd_mm: float = 2.0, threshold: float = 0.2) -> float:
    """Fraction of reference voxels with ref > threshold * max(ref) that have
    gamma <= 1.  Arrays are (nz, ny, nx); voxel_mm = (dx, dy, dz) in mm."""
    ref = np.asarray(ref, dtype=np.float64)
    ev = np.asarray(ev, dtype=np.float64)
    dmax = ref.max()
    dD = dd_frac * dmax
    idx = np.argwhere(ref > threshold * dmax)  # (k, 3) in (z, y, x)
    if len(idx) == 0:
        return 1.0
    d_ref = ref[tuple(idx.T)]
    dx, dy, dz = voxel_mm
    h = dd_mm / 10.0
    n = int(np.ceil(dd_mm / h))
    g = np.arange(-n, n + 1) * h
    oz, oy, ox = np.meshgrid(g, g, g, indexing="ij")
    r2 = (ox ** 2 + oy ** 2 + oz ** 2).ravel()
    keep = r2 <= dd_mm ** 2
    offs = np.stack([oz.ravel()[keep] / dz, oy.ravel()[keep] / dy, ox.ravel()[keep] / dx], 1)
    r2 = r2[keep]
    order = np.argsort(r2)
    offs, r2 = offs[order], r2[order]
    active = np.ones(len(idx), dtype=bool)
    pts = idx.astype(np.float64)
    for o, rr in zip(offs, r2):
        a = np.nonzero(active)[0]
        if a.size == 0:
            break
        coords = (pts[a] + o).T
        val = map_coordinates(ev, coords, order=1, mode="nearest")
        g2 = rr / dd_mm ** 2 + ((val - d_ref[a]) / dD) ** 2
        active[a[g2 <= 1.0]] = False
    return float(1.0 - active.mean())

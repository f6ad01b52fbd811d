"""Phantom set-up on the device: the per-material maximum densities and the
Woodcock majorants of a phantom (GPUMCD §II.A, the photon mu_max; §II.B.3,
the electron Sigma_hat) equal their definitions restated on the host, bit for
bit, from the phantom and the library's own cross-section tables.

- The maximum density of material m is the largest density among the
  phantom's voxels of material m, after quantisation to 2^-24 g/cm^3.
- The photon majorant at grid point i is max over materials of
  rho_max[m] * mu_m[i].
- The electron majorant at i is the running maximum over j <= i of
  max_m rho_max[m] * Sigma_hard,m[j].

Maxima and single float32 products are exact, so the comparison is exact. The
phantoms are sized to span several CTAs with a ragged tail, and the densities
spread so that the reductions across warps and CTAs decide the result.
"""
import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu
G = 512


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def host_rho_max(ph: W.Phantom, n_mat: int) -> np.ndarray:
    r = np.ascontiguousarray(ph.rho, dtype=np.float32).ravel()
    m = np.ascontiguousarray(ph.mat).ravel()
    q = np.rint(r * np.float32(2.0 ** 24)).astype(np.float64)  # round to nearest even
    q = np.clip(q, 1, 2 ** 28 - 1).astype(np.uint32)
    val = q.astype(np.float32) * np.float32(2.0 ** -24)
    out = np.zeros(g.MAX_MATERIALS, dtype=np.float32)
    for k in range(n_mat):
        sel = m == k
        if sel.any():
            out[k] = val[sel].max()
    return out


def host_majorants(ctx, rho_max: np.ndarray, n_mat: int) -> np.ndarray:
    tp = ctx.get_tables(0).reshape(g.MAX_MATERIALS, 3, G)
    te = ctx.get_tables(1).reshape(g.MAX_MATERIALS, 4, G)
    mp = np.zeros(G, dtype=np.float32)
    me = np.zeros(G, dtype=np.float32)
    for k in range(n_mat):
        r = np.float32(rho_max[k])
        if r <= 0:
            continue
        mp = np.maximum(mp, r * tp[k, 0])
        me = np.maximum(me, r * te[k, 1])
    return np.concatenate([mp, np.maximum.accumulate(me)])


def spread_phantom(dims, seed):
    """Every voxel its own material (all loaded ones) and density, from a
    seeded generator: the maxima sit in random voxels."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    mat = rng.integers(0, len(W.MATERIALS), size=(nz, ny, nx)).astype(np.uint8)
    rho = rng.uniform(0.001, 15.9, size=(nz, ny, nx)).astype(np.float32)
    return W.Phantom((nx, ny, nz), (0.3, 0.3, 0.3), mat, rho)


CASES = {
    "noise_37": lambda: W.smoothed_noise(37, 0.5, np.random.default_rng(11)),
    "spread_61x47x33": lambda: spread_phantom((61, 47, 33), 12),
    "spread_ragged_300x7x5": lambda: spread_phantom((300, 7, 5), 13),
    "water_only": lambda: W.homogeneous((16, 9, 5), 0.5, W.MAT_WATER, 1.0),
    "one_voxel_bone": lambda: W.homogeneous((1, 1, 1), 0.5, W.MAT_BONE, 1.85),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_majorants_equal_their_definition(ctx, name):
    ph = CASES[name]()
    n_mat = len(W.MATERIALS)
    pid = ctx.create_phantom(ph)
    try:
        maj, rho_max = ctx.debug_majorants(pid)
    finally:
        ctx.destroy_phantom(pid)
    want_rho = host_rho_max(ph, n_mat)
    assert np.array_equal(rho_max.view(np.uint32), want_rho.view(np.uint32))
    want = host_majorants(ctx, want_rho, n_mat)
    assert np.array_equal(maj.view(np.uint32), want.view(np.uint32))
    assert np.all(np.diff(maj[G:]) >= 0)  # the electron majorant never falls with energy


def test_one_bad_voxel_rejects_the_phantom(ctx):
    ph = spread_phantom((61, 47, 33), 14)
    ph.rho[20, 30, 40] = 16.5  # outside the packed density range
    with pytest.raises(g.GpumcdError) as e:
        ctx.create_phantom(ph)
    assert e.value.status == g.ERR_INVALID_ARG
    ph.rho[20, 30, 40] = 1.0
    ph.mat[3, 4, 5] = len(W.MATERIALS)  # a material that was never loaded
    with pytest.raises(g.GpumcdError) as e:
        ctx.create_phantom(ph)
    assert e.value.status == g.ERR_INVALID_ARG

"""Dose parity on the paper's second and third geometries (GPUMCD §III.A): a
lung box in water, and slabs of soft tissue, lung and bone, each in its
electron and photon arrangement.  The grids are the paper's own 64^3 at
0.5 cm (the timing workload uses 128^3 at 0.25 cm over the same 32 cm).

The histories are cut so that the oracle finishes in seconds. The
bar is the one of the other parity tests:
- >= 99% of voxels above 10% of D_max within 3 combined sigma;
- an exact integer ledger;
- per-history rates of real events (electron steps, real hard events, real
  photon interactions) within a few per cent.

Fictitious events are not compared. Their count depends on how each side
tabulates its majorant: the GPU uses its 512-point grid. Any valid majorant
leaves the real-event rates and the dose unchanged (Woodcock tracking,
§II.A, §II.B.3). The share of fictitious events, which the bone slab's
density drives up, is a measured output of `bench.py --workload geoms`.
"""
import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests._stats import three_sigma_pass_rate
from tests.gpu_common import ledger_exact, need_gpu, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = g.engine(0, mats=W.MATERIALS_PAPER)
    yield c
    c.close()


CASES = [
    ("geom2", W.ELECTRON, 20_000),
    ("geom2", W.PHOTON, 60_000),
    ("geom3", W.ELECTRON, 20_000),
    ("geom3", W.PHOTON, 60_000),
]


@pytest.mark.parametrize("geom,particle,n", CASES, ids=[f"{c[0]}-{'e' if c[1] == W.ELECTRON else 'g'}" for c in CASES])
def test_paper_geometry_parity(ctx, geom, particle, n):
    plan = getattr(W, geom)(particle, n_histories=n, n=64, voxel_cm=0.5)
    gpu = run_gpu(ctx, plan)
    ora = run_oracle(plan, mats=W.MATERIALS_PAPER)
    assert ledger_exact(gpu.stats)
    ph = plan.phantom
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert mask.sum() > 100
    rate = three_sigma_pass_rate(gpu.dose, gpu.sigma, do, so, mask)
    assert rate >= 0.99, rate
    st, os_ = gpu.stats, ora.stats
    assert st["n_electron_steps"] / n == pytest.approx(os_["n_e_steps"] / n, rel=0.03)
    assert st["n_hard_real"] / n == pytest.approx(os_["n_hard_real"] / n, rel=0.05)
    assert st["n_photon_real"] / n == pytest.approx(os_["n_photon_real"] / n, rel=0.05)

"""The GPU's uncertainty estimate and the run to a target uncertainty
(GPUMCD §II.D).

The GPU estimates sigma from W interleaved batch tallies; the oracle from
history-by-history moments.  Both estimate the standard error of the same mean
dose, so on the same phantom and beam at the same history count their sigmas
agree voxel by voxel up to the estimators' own scatter: the median of
sigma_gpu / sigma_oracle over the voxels above 20% of D_max is 1 within a few
percent, and the z-scores (D_gpu - D_ora) / sqrt(sigma_gpu^2 + sigma_ora^2)
spread as a unit normal.  An estimator that is off by a constant factor (a
missing sqrt(W / (W - 1)), a variance of the sum instead of the mean) fails
both.

gpumcd_simulate with target_rel_unc > 0 runs rounds of n histories until
s_0.5 (mean sigma/D over voxels above half of D_max) reaches the target; its
dose equals, bit for bit, that of one plain run of the same history count.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.conftest import host_cores
from tests.gpu_common import ledger_exact, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def _gpu(ctx, ph, src, n, seed, n_batches):
    import torch
    pid = ctx.create_phantom(ph)
    p = ctx.plan_open(pid, src, seed, n_batches)
    ctx.run([p], [n])
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(d)
    st = ctx.plan_result(p, 0.5, d.data_ptr(), s.data_ptr())
    ctx.plan_close(p)
    ctx.destroy_phantom(pid)
    return d.cpu().numpy(), s.cpu().numpy(), st


CASES = {
    "electron_field": (W.homogeneous((24, 24, 40), 0.5, W.MAT_WATER, 1.0),
                       W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=10.0, center_cm=(6.0, 6.0), field_cm=4.0),
                       200_000),
    "photon_slabs": (W.z_slabs((20, 20, 48), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                                   (6.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)]),
                     W.Source(W.PHOTON, W.BEAM_SQUARE, energy=6.0, center_cm=(5.0, 5.0), field_cm=5.0),
                     1_000_000),
}


_ORACLE = {}


def _oracle(case):
    if case not in _ORACLE:
        ph, src, n = CASES[case]
        ora = oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, n, 6, processes=host_cores())
        _ORACLE[case] = (ora.dose_gy(ph), ora.sigma_gy(ph))
    return _ORACLE[case]


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_batches", [16, 32])
def test_gpu_sigma_matches_oracle_sigma(ctx, case, n_batches):
    ph, src, n = CASES[case]
    dg, sg, st = _gpu(ctx, ph, src, n, 5, n_batches)
    assert ledger_exact(st)
    do, so = _oracle(case)
    mask = do > 0.2 * do.max()
    assert mask.sum() > 100
    ratio = sg[mask] / so[mask]
    # a batch sigma with W - 1 degrees of freedom scatters by ~1/sqrt(2(W-1)); its median is ~1
    assert float(np.median(ratio)) == pytest.approx(1.0, abs=0.05), float(np.median(ratio))
    z = (dg - do)[mask] / np.sqrt(sg ** 2 + so ** 2)[mask]
    assert abs(float(np.mean(z))) < 0.2, float(np.mean(z))
    assert 0.85 < float(np.std(z)) < 1.15, float(np.std(z))
    assert float(np.mean(np.abs(z) <= 3.0)) >= 0.99


def test_run_to_uncertainty_through_the_c_abi(ctx):
    import torch
    ph = W.homogeneous((24, 24, 40), 0.5, W.MAT_WATER, 1.0)
    src = W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=8.0, center_cm=(6.0, 6.0), field_cm=4.0)
    pid = ctx.create_phantom(ph)
    n, target, seed = 20_000, 0.02, 77
    r = ctx.simulate(pid, src, n, seed, target_rel_unc=target, nvox=ph.nvox)
    st = r.stats
    total = st["histories"]
    assert ledger_exact(st)
    assert total % n == 0 and total >= 2 * n  # more than one round was needed
    assert st["s_thr"] <= target
    # one round fewer had not reached the target
    p = ctx.plan_open(pid, src, seed, 32)
    ctx.run([p], [total - n])
    assert ctx.plan_result(p, 0.5)["s_thr"] > target
    ctx.plan_close(p)
    # the same history count in one plain run gives the same dose, bit for bit
    p = ctx.plan_open(pid, src, seed, 32)
    ctx.run([p], [total])
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(d)
    st2 = ctx.plan_result(p, 0.5, d.data_ptr(), s.data_ptr())
    assert np.array_equal(d.cpu().numpy(), r.dose)
    assert np.array_equal(s.cpu().numpy(), r.sigma)
    assert st2["s_thr"] == pytest.approx(st["s_thr"], rel=1e-12)
    assert st2["e_deposited"] == st["e_deposited"]
    ctx.plan_close(p)
    ctx.destroy_phantom(pid)

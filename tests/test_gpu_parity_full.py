"""Parity at the configs' full sizes, in the benchmark's launch configuration.

The oracle cannot run the full history counts in seconds, so at full phantom
sizes the comparisons use what holds at any size:
- per voxel, GPU at full histories against the oracle at fewer histories,
  each with its own sigma (>= 99% of voxels above 10% of D_max within 3
  combined sigma);
- depth-dose curves averaged over the central square, with the sigma of each
  average taken from K independent sub-runs on each side (neighbouring voxels
  are correlated, so per-voxel sigmas do not add up);
- the exact integer energy ledger.
Where the oracle can reach a reference noise under 1% of D_max in the
high-dose region, the gamma index (2%/2 mm, voxels above 20% of D_max) must
pass for >= 98% of voxels: C1 with both sides at 4e6 histories, the C2
beams on the paper's own 64^3 grid of 0.5 cm voxels, and the C3 beam and
slabs on 32^3 voxels of 1 cm.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._gamma import gamma_pass_rate
from tests._stats import three_sigma_pass_rate
from tests.conftest import host_cores
from tests.gpu_common import ledger_exact, make_ctx

pytestmark = pytest.mark.gpu
K = 12


def _gpu_runs(ctx, plan, n_total, k=K, seed0=100):
    """k independent GPU runs (seeds seed0..seed0+k-1) of n_total/k histories."""
    import torch
    pid = ctx.create_phantom(plan.phantom)
    doses, sigmas, stats = [], [], []
    for i in range(k):
        p = ctx.plan_open(pid, plan.source, seed0 + i, 32)
        ctx.run([p], [n_total // k])
        d = torch.zeros(plan.phantom.nvox, dtype=torch.float64, device="cuda")
        s = torch.zeros_like(d)
        st = ctx.plan_result(p, 0.5, d.data_ptr(), s.data_ptr())
        doses.append(d.cpu().numpy())
        sigmas.append(s.cpu().numpy())
        stats.append(st)
        ctx.plan_close(p)
    ctx.destroy_phantom(pid)
    return np.array(doses), np.array(sigmas), stats


def _oracle_runs(plan, n_total, k=K, seed=500):
    return oracle.simulate_parts(W.MATERIALS, W.DEFAULT_PHYSICS, plan.phantom, plan.source, n_total,
                                 seed, k, processes=host_cores())


def _combine_oracle(runs, ph):
    n = sum(r.n_histories for r in runs)
    s1 = sum(r.sum_e for r in runs)
    s2 = sum(r.sum_e2 for r in runs)
    tot = oracle.OracleResult(n, s1, s2, {})
    return tot.dose_gy(ph), tot.sigma_gy(ph)


def _pdd(d, ph, half_cm):
    nx, ny, nz = ph.dims
    vx = ph.voxel_cm[0]
    c = nx // 2
    h = max(1, int(round(half_cm / vx)))
    vol = d.reshape(-1, nz, ny, nx) if d.ndim == 2 else d.reshape(nz, ny, nx)
    if d.ndim == 2:
        return vol[:, :, c - h:c + h, c - h:c + h].mean(axis=(2, 3))
    return vol[:, c - h:c + h, c - h:c + h].mean(axis=(1, 2))


def _curve_parity(g_runs, o_runs_dose, frac=0.1):
    """3-sigma agreement of two curves, each estimated as the mean of K runs."""
    gm, om = g_runs.mean(0), o_runs_dose.mean(0)
    gs = g_runs.std(0, ddof=1) / np.sqrt(len(g_runs))
    os_ = o_runs_dose.std(0, ddof=1) / np.sqrt(len(o_runs_dose))
    mask = om > frac * om.max()
    ok = np.abs(gm - om)[mask] <= 3 * np.sqrt(gs ** 2 + os_ ** 2)[mask]
    return float(ok.mean()), int(mask.sum())


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_c1_full_size_gamma_and_three_sigma(ctx):
    # 4e6 histories on both sides keep the statistical noise of the few
    # significant voxels of a pencil beam well under the 2% dose criterion
    plan = W.config1(n_histories=4_000_000)
    g = _gpu_runs(ctx, plan, plan.n_histories, k=1, seed0=1)
    ora = oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, plan.phantom, plan.source, plan.n_histories, 77,
                          processes=host_cores())
    ph = plan.phantom
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    dg, sg = g[0][0], g[1][0]
    assert ledger_exact(g[2][0])
    mask = do > 0.1 * do.max()
    assert three_sigma_pass_rate(dg, sg, do, so, mask) >= 0.99
    vox_mm = tuple(10 * v for v in ph.voxel_cm)
    rate = gamma_pass_rate(do.reshape(32, 32, 32), dg.reshape(32, 32, 32), vox_mm)
    assert rate >= 0.98, (rate, int((do > 0.2 * do.max()).sum()))


@pytest.mark.parametrize("particle,n_gpu,n_ora", [(W.ELECTRON, 1_000_000, 36_000),
                                                  (W.PHOTON, 4_000_000, 120_000)])
def test_c2_full_size(ctx, particle, n_gpu, n_ora):
    plan = W.config2(particle)
    ph = plan.phantom
    gd, gs, gst = _gpu_runs(ctx, plan, n_gpu)
    assert all(ledger_exact(s) for s in gst)
    oruns = _oracle_runs(plan, n_ora)
    od = np.array([r.dose_gy(ph) for r in oruns])
    # per voxel: full-history GPU against the pooled oracle
    do, so = _combine_oracle(oruns, ph)
    dg = gd.mean(0)
    sg = gd.std(0, ddof=1) / np.sqrt(K)
    mask = do > 0.1 * do.max()
    assert three_sigma_pass_rate(dg, sg, do, so, mask) >= 0.99
    # central-axis depth dose over the central 1 x 1 cm
    rate, n = _curve_parity(_pdd(gd, ph, 0.5), _pdd(od, ph, 0.5))
    assert n > 10 and rate >= 0.97, rate


def test_c3_full_size_slabs_spectrum(ctx):
    plan = W.config3(n_histories=10_000_000)
    ph = plan.phantom
    gd, gs, gst = _gpu_runs(ctx, plan, plan.n_histories)
    assert all(ledger_exact(s) for s in gst)
    oruns = _oracle_runs(plan, 240_000)
    od = np.array([r.dose_gy(ph) for r in oruns])
    do, so = _combine_oracle(oruns, ph)
    dg = gd.mean(0)
    sg = gd.std(0, ddof=1) / np.sqrt(K)
    mask = do > 0.1 * do.max()
    assert three_sigma_pass_rate(dg, sg, do, so, mask) >= 0.99
    rate, n = _curve_parity(_pdd(gd, ph, 1.0), _pdd(od, ph, 1.0))
    assert n > 10 and rate >= 0.97, rate
    # per slab (water, bone, lung, water): the mean dose inside the central
    # 8 x 8 cm averages ~1e5 voxels, so it checks the heterogeneity handling
    # far more sharply than single voxels; the standard errors come from the
    # spread of the K independent runs on each side
    nx, ny, nz = ph.dims
    mats = ph.mat[:, 0, 0]
    bounds = [0] + [z for z in range(1, nz) if mats[z] != mats[z - 1]] + [nz]
    c, h = nx // 2, 20
    for z0, z1 in zip(bounds[:-1], bounds[1:]):
        def slab(d):
            return d.reshape(-1, nz, ny, nx)[:, z0:z1, c - h:c + h, c - h:c + h].mean(axis=(1, 2, 3))
        g_m, o_m = slab(gd), slab(od)
        se = np.sqrt(g_m.var(ddof=1) / len(g_m) + o_m.var(ddof=1) / len(o_m))
        assert abs(g_m.mean() - o_m.mean()) <= 3.5 * se, (z0, z1, g_m.mean(), o_m.mean(), se)


@pytest.mark.parametrize("particle,n_gpu,n_ora", [(W.ELECTRON, 30_000_000, 6_000_000),
                                                  (W.PHOTON, 180_000_000, 36_000_000)])
def test_c2_beams_gamma_on_the_paper_grid(ctx, particle, n_gpu, n_ora):
    """The timing-case beams (15 MeV, 10 x 10 cm^2) on the paper's own grid for
    its gamma comparisons, 64^3 water voxels of 0.5 cm (GPUMCD §III.A, Geom1):
    gamma 2% / 2 mm over voxels above 20% of D_max passes for >= 98% of them,
    with the oracle as the reference.  The oracle runs enough histories that its
    own noise in the high-dose region is under 0.8% of D_max (the gamma index
    has no term for the reference's noise: at 1.2-1.5% noise a flawless
    evaluation would fail ~10% of the flat high-dose voxels), the GPU five
    times more."""
    plan = W.config2(particle, n=64, voxel_cm=0.5)
    ph = plan.phantom
    gd, gs, gst = _gpu_runs(ctx, plan, n_gpu, k=1, seed0=3)
    assert ledger_exact(gst[0])
    ora = oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, ph, plan.source, n_ora, 91,
                          processes=host_cores())
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    high = do > 0.5 * do.max()
    noise = float(np.median(so[high] / do.max()))
    dg, sg = gd[0], gs[0]
    rate = gamma_pass_rate(do.reshape(64, 64, 64), dg.reshape(64, 64, 64), (5.0, 5.0, 5.0))
    assert noise < 0.008, (noise, rate)
    assert three_sigma_pass_rate(dg, sg, do, so, do > 0.1 * do.max()) >= 0.99
    assert rate >= 0.98, (rate, noise)


def test_c3_slabs_gamma_on_a_coarse_grid(ctx):
    """The slab configuration's beam and phantom (a 6 MV-like spectrum on a
    10 x 10 cm^2 field into water / bone / lung / water slabs of 3 / 2 / 6 /
    rest cm) on 32^3 voxels of 1 cm: gamma 2% / 2 mm over voxels above 20% of
    D_max passes for >= 98% of them, with the oracle as the reference.  At
    the configuration's own 0.2 cm voxels the oracle cannot reach a reference
    noise under 1% of D_max (a photon beam's voxels see few interactions);
    1 cm voxels collect 125 times more events each, and 3.2e7 oracle
    histories bring the noise in the high-dose region under 0.8%."""
    plan = W.config3(n=32, voxel_cm=1.0)
    ph = plan.phantom
    gd, gs, gst = _gpu_runs(ctx, plan, 160_000_000, k=1, seed0=31)
    assert ledger_exact(gst[0])
    ora = oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, ph, plan.source, 32_000_000, 131,
                          processes=host_cores())
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    noise = float(np.median(so[do > 0.5 * do.max()] / do.max()))
    dg, sg = gd[0], gs[0]
    rate = gamma_pass_rate(do.reshape(32, 32, 32), dg.reshape(32, 32, 32), (10.0, 10.0, 10.0))
    assert noise < 0.008, (noise, rate)
    assert three_sigma_pass_rate(dg, sg, do, so, do > 0.1 * do.max()) >= 0.99
    assert rate >= 0.98, (rate, noise)

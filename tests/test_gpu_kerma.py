"""The photon-only mode (GPUMCD_LAUNCH_KERMA, the "photon-only fast mode" of
the paper's outlook, §V): electrons deposit their kinetic energy in the voxel
where they are created and are not transported.  Parity is against the
oracle's own KERMA mode, on the same seeded inputs, with the bar of the other
parity tests (>= 99% of voxels above 10% of D_max within 3 combined sigma,
exact ledger, matching photon interaction rates)."""
import numpy as np
import pytest

import oracle
import paper_1101_1245_gb300 as g
import workloads as W
from tests._stats import three_sigma_pass_rate
from tests.gpu_common import ledger_exact, make_ctx, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx(flags=g.LAUNCH_KERMA)
    yield c
    c.close()


def _slabs():
    ph = W.z_slabs((20, 20, 48), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                        (6.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    src = W.Source(W.PHOTON, W.BEAM_SQUARE, energy=15.0, center_cm=(5.0, 5.0), field_cm=4.0)
    return W.Plan("kerma_slabs_15MeV", ph, src, 200_000, 21)


@pytest.mark.parametrize("make", [lambda: W.config1(n_histories=200_000), _slabs], ids=["c1", "slabs15"])
def test_kerma_parity(ctx, make):
    plan = make()
    gpu = run_gpu(ctx, plan)
    ora = run_oracle(plan, flags=oracle.FLAG_KERMA)
    assert ledger_exact(gpu.stats)
    assert gpu.stats["n_electron_steps"] == 0 and gpu.stats["n_hard_real"] == 0
    ph = plan.phantom
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert mask.sum() > 30
    rate = three_sigma_pass_rate(gpu.dose, gpu.sigma, do, so, mask)
    assert rate >= 0.99, rate
    n = plan.n_histories
    for k in ("n_photon_real", "n_compton", "n_pair"):
        if ora.stats[k] > 1000:
            assert gpu.stats[k] / n == pytest.approx(ora.stats[k] / n, rel=0.03), k


def test_kerma_electron_beam_deposits_at_entry(ctx):
    """A primary electron deposits its whole energy in its entry voxel (z = 0)."""
    ph = W.homogeneous((10, 8, 6), 0.5, W.MAT_WATER, 1.0)
    src = W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=6.0, center_cm=(2.5, 2.0), field_cm=2.0)
    r = run_gpu(ctx, W.Plan("kerma_e", ph, src, 5000, 3))
    assert r.stats["e_deposited"] == r.stats["e_incident"] == 5000 * round(6.0 * 2 ** 26)
    d = r.dose.reshape(6, 8, 10)
    assert d[0].sum() > 0 and np.all(d[1:] == 0)
    assert r.stats["n_electron_steps"] == 0


def test_kerma_off_restores_transport():
    """The flag selects the photon-only kernel; clearing it runs the transport
    kernel again, with the same result bit for bit."""
    plan = W.config1(n_histories=20_000)
    c = make_ctx()
    a = run_gpu(c, plan)
    c.set_launch(flags=g.LAUNCH_KERMA)
    k = run_gpu(c, plan)
    c.set_launch(flags=0)
    b = run_gpu(c, plan)
    c.close()
    assert np.array_equal(a.dose, b.dose) and a.stats["n_electron_steps"] > 0
    assert k.stats["n_electron_steps"] == 0 and not np.array_equal(a.dose, k.dose)

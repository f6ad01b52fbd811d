"""Phase-space sources (GPUMCD_BEAM_PHASE_SPACE, the phase-space sources of the
paper's outlook, §V): history h starts as record h mod n of a caller-supplied
list.  Also the energy grouping of polyenergetic sources (§IV), which both
phase spaces and spectra take.  Parity is against the oracle's own phase-space source on the same
seeded records, with the bar of the other parity tests:
- >= 99% of voxels above 10% of D_max within 3 combined sigma;
- an exact integer ledger;
- an incident energy equal to the records' energies taken in turn, in quanta."""
import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests._stats import three_sigma_pass_rate
from tests.gpu_common import ledger_exact, make_ctx, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
Q = 2.0 ** -26


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def _incident_quanta(src, n):
    e = src.phase_space[:, 6].astype(np.float32)
    q = np.rint(e.astype(np.float32) * np.float32(2 ** 26)).astype(np.uint64)
    k = len(e)
    return int(q.sum()) * (n // k) + int(q[: n % k].sum())


CASES = [
    ("electron_water", W.ELECTRON, lambda: W.homogeneous((32, 32, 40), 0.5, W.MAT_WATER, 1.0), 20_000),
    ("photon_slabs", W.PHOTON, lambda: W.z_slabs((32, 32, 48), 0.5, [(3.0, W.MAT_WATER, 1.0),
                                                                       (2.0, W.MAT_BONE, 1.85),
                                                                       (6.0, W.MAT_LUNG, 0.26),
                                                                       (1e9, W.MAT_WATER, 1.0)]), 100_000),
]


@pytest.mark.parametrize("name,particle,make_ph,n", CASES, ids=[c[0] for c in CASES])
def test_phase_space_parity(ctx, name, particle, make_ph, n):
    ph = make_ph()
    src = W.point_source_phase_space(particle, ph, 997, seed=21, field_cm=8.0)
    plan = W.Plan(name, ph, src, n, 31)
    gpu = run_gpu(ctx, plan)
    ora = run_oracle(plan)
    assert ledger_exact(gpu.stats)
    assert gpu.stats["e_incident"] == _incident_quanta(src, n)
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert mask.sum() > 100
    rate = three_sigma_pass_rate(gpu.dose, gpu.sigma, do, so, mask)
    assert rate >= 0.99, rate
    key = "n_electron_steps" if particle == W.ELECTRON else "n_photon_real"
    okey = "n_e_steps" if particle == W.ELECTRON else "n_photon_real"
    assert gpu.stats[key] / n == pytest.approx(ora.stats[okey] / n, rel=0.03)


def test_phase_space_of_the_pencil_matches_the_pencil(ctx):
    """Records that all list the pencil beam's primary give the pencil run's
    dose within statistics (a separately compiled kernel, the same physics)."""
    ph = W.homogeneous((24, 24, 30), 0.5, W.MAT_WATER, 1.0)
    pen = W.pencil(W.PHOTON, 3.0, 6.0, 6.0)
    rec = np.repeat(np.array([[6.0, 6.0, 0.0, 0.0, 0.0, 1.0, 3.0]]), 3, axis=0)
    phs = W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=rec)
    a = run_gpu(ctx, W.Plan("pencil", ph, pen, 100_000, 5))
    b = run_gpu(ctx, W.Plan("phsp", ph, phs, 100_000, 5))
    assert a.stats["e_incident"] == b.stats["e_incident"]
    mask = a.dose > 0.1 * a.dose.max()
    assert three_sigma_pass_rate(b.dose, b.sigma, a.dose, a.sigma, mask) >= 0.99


def test_phase_space_validation(ctx):
    ph = W.homogeneous((8, 8, 8), 0.5, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    try:
        bad = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 25.0]])  # above e_max
        with pytest.raises(g.GpumcdError) as e:
            ctx.plan_open(pid, W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=bad), 1, 16)
        assert e.value.status == g.ERR_INVALID_ARG
        zero = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 2.0]])  # no direction
        with pytest.raises(g.GpumcdError) as e:
            ctx.plan_open(pid, W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=zero), 1, 16)
        assert e.value.status == g.ERR_INVALID_ARG
        good = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 2.0]])
        plan = ctx.plan_open(pid, W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=good), 1, 16)
        ctx.set_launch(flags=g.LAUNCH_KERMA)  # no phase-space variant of the photon-only kernel
        with pytest.raises(g.GpumcdError) as e:
            ctx.run([plan], [64])
        assert e.value.status == g.ERR_INVALID_ARG
        ctx.set_launch(flags=0)
        ctx.run([plan], [64])
        assert ctx.plan_result(plan, 0.5)["histories"] == 64
        ctx.plan_close(plan)
    finally:
        ctx.destroy_phantom(pid)


def _tied_phase_space(ph, n, seed):
    """Records in random order whose energies take only 7 values, so that the
    stable order of ties decides which record each history takes."""
    src = W.point_source_phase_space(W.PHOTON, ph, n, seed=seed, field_cm=6.0)
    rng = np.random.default_rng(seed + 1)
    src.phase_space[:, 6] = rng.choice([0.3, 0.8, 1.25, 2.0, 3.5, 6.0, 9.0], size=n)
    return src


def test_grouped_phase_space_equals_ungrouped(ctx):
    """GPUMCD_ENERGY_GROUPED on a phase space orders each launch's claims by
    the records' energies and leaves the sample alone: history h starts as
    record h mod n of the list as given.  The tally, the ledger and every
    counter equal, bit for bit, those of the ungrouped plan (997 records with
    7 distinct energies in random order), split into ragged runs or not, and
    also for fewer histories than records, where a list sorted by energy would
    start only the highest-energy records."""
    ph = W.homogeneous((24, 24, 30), 0.5, W.MAT_WATER, 1.0)
    src = _tied_phase_space(ph, 997, 41)
    grouped = W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=src.phase_space,
                       energy_grouping=W.ENERGY_GROUPED)
    for runs in ([30_011], [10_007, 20_004], [300]):
        n = sum(runs)
        a = _phsp_kernel_runs(ctx, ph, grouped, 9, runs)
        b = _phsp_kernel_runs(ctx, ph, src, 9, [n])
        assert np.array_equal(a[0].view(np.uint64), b[0].view(np.uint64)), runs
        assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64)), runs
        for key in ("e_incident", "e_deposited", "e_escaped", "e_rest", "n_photon_real", "n_electron_steps",
                    "n_compton", "n_photo", "n_pair", "n_moller", "n_brem"):
            assert a[2][key] == b[2][key], (runs, key)
        assert a[2]["e_incident"] == _incident_quanta(src, n)
        assert ledger_exact(a[2])


def test_grouped_by_energy_parity(ctx):
    """A grouped polyenergetic photon phase space against the oracle (for
    which grouping changes nothing): the parity bar of the other phase-space
    tests."""
    ph = W.z_slabs((32, 32, 48), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                       (6.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    src = W.polyenergetic_phase_space(W.PHOTON, ph, 1009, seed=23)
    src.energy_grouping = W.ENERGY_GROUPED
    plan = W.Plan("grouped_slabs", ph, src, 100_000, 37)
    gpu = run_gpu(ctx, plan)
    ora = run_oracle(plan)
    assert ledger_exact(gpu.stats)
    assert gpu.stats["e_incident"] == _incident_quanta(src, 100_000)
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert mask.sum() > 100
    assert three_sigma_pass_rate(gpu.dose, gpu.sigma, do, so, mask) >= 0.99
    assert gpu.stats["n_photon_real"] / 100_000 == pytest.approx(ora.stats["n_photon_real"] / 100_000, rel=0.03)


def test_energy_grouping_is_validated(ctx):
    ph = W.homogeneous((8, 8, 8), 0.5, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    try:
        rec = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 2.0]])
        with pytest.raises(g.GpumcdError) as e:
            ctx.plan_open(pid, W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=rec, energy_grouping=2), 1, 16)
        assert e.value.status == g.ERR_INVALID_ARG
        bad = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 2.0], [1.0, 1.0, 0.0, 0.0, 0.0, 1.0, np.nan]])
        with pytest.raises(g.GpumcdError) as e:  # a record that is not finite
            ctx.plan_open(pid, W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=bad,
                                        energy_grouping=W.ENERGY_GROUPED), 1, 16)
        assert e.value.status == g.ERR_INVALID_ARG
    finally:
        ctx.destroy_phantom(pid)


def _mean_energy(edges, w):
    return float(np.sum(np.asarray(w) * 0.5 * (edges[:-1] + edges[1:])) / np.sum(w))


def _phsp_kernel_runs(ctx, ph, src, seed, runs):
    """A plan run as `runs` on the phase-space kernel: a phase space runs there
    by itself; beside any other source, in each launch, a one-record phase
    space of the same particle type runs one history (the launch's event
    counters, which go to its first plan, then include that history).
    Returns the plan's dose, sigma and stats."""
    import torch
    pid = ctx.create_phantom(ph)
    dummy = None
    if src.beam != W.BEAM_PHASE_SPACE:
        rec = np.array([[0.5 * ph.extent_cm[0], 0.5 * ph.extent_cm[1], 0.0, 0.0, 0.0, 1.0, 1.0]])
        dummy = ctx.plan_open(pid, W.Source(src.particle, W.BEAM_PHASE_SPACE, phase_space=rec), 1, 8)
    plan = ctx.plan_open(pid, src, seed, 16)
    for n in runs:
        ctx.run([plan] if dummy is None else [plan, dummy], [n] if dummy is None else [n, 1])
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(d)
    st = ctx.plan_result(plan, 0.5, d.data_ptr(), s.data_ptr())
    ctx.plan_close(plan)
    if dummy is not None:
        ctx.plan_close(dummy)
    ctx.destroy_phantom(pid)
    return d.cpu().numpy(), s.cpu().numpy(), st


def test_grouped_spectrum_equals_ungrouped_and_the_oracle(ctx):
    """A 6 MV-like photon spectrum grouped by energy (§IV): its launches claim
    the histories in decreasing order of their energy, and each history draws
    what it draws ungrouped.  On the same (phase-space) kernel the grouped and
    ungrouped tallies are equal bit for bit, split into runs or not; the
    grouped one passes the oracle's 3-sigma test with an exact ledger."""
    edges, w = W.synthetic_6mv_spectrum()
    ph = W.z_slabs((32, 32, 48), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                       (6.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    src = W.Source(W.PHOTON, W.BEAM_SQUARE, center_cm=(8.0, 8.0), field_cm=8.0, spectrum_edges=edges,
                   spectrum_weights=w, energy_grouping=W.ENERGY_GROUPED)
    plain = W.Source(W.PHOTON, W.BEAM_SQUARE, center_cm=(8.0, 8.0), field_cm=8.0, spectrum_edges=edges,
                     spectrum_weights=w)
    n = 100_000
    dg, sg, st = _phsp_kernel_runs(ctx, ph, src, 43, [n])
    du, su, stu = _phsp_kernel_runs(ctx, ph, plain, 43, [n])
    dsplit, _, _ = _phsp_kernel_runs(ctx, ph, src, 43, [30_011, 50_000, n - 80_011])
    assert np.array_equal(dg, du) and np.array_equal(sg, su) and np.array_equal(dg, dsplit)
    assert st["e_incident"] == stu["e_incident"]
    assert ledger_exact(st)
    ora = run_oracle(W.Plan("grouped_spectrum", ph, src, n, 43))
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert mask.sum() > 100
    assert three_sigma_pass_rate(dg, sg, do, so, mask) >= 0.99
    assert st["n_photon_real"] / n == pytest.approx(ora.stats["n_photon_real"] / n, rel=0.03)


def test_grouping_leaves_a_monoenergetic_beam_unchanged(ctx):
    """A monoenergetic beam has nothing to group: its tallies are bit-identical
    with and without the flag (the production kernel runs both)."""
    ph = W.homogeneous((16, 16, 24), 0.5, W.MAT_WATER, 1.0)
    a = run_gpu(ctx, W.Plan("mono", ph, W.pencil(W.ELECTRON, 6.0, 4.0, 4.0), 20_000, 3))
    src = W.pencil(W.ELECTRON, 6.0, 4.0, 4.0)
    src.energy_grouping = W.ENERGY_GROUPED
    b = run_gpu(ctx, W.Plan("mono_grouped", ph, src, 20_000, 3))
    assert np.array_equal(a.dose.view(np.uint64), b.dose.view(np.uint64))
    assert a.stats["n_electron_steps"] == b.stats["n_electron_steps"]


def test_grouped_spectrum_runs_the_phase_space_kernel(ctx):
    """A grouped spectral plan is drawn by the phase-space instantiation, so the
    photon-only flag (which has no such instantiation) is refused for it, and
    accepted again for the same spectrum ungrouped."""
    edges, w = W.synthetic_6mv_spectrum(n_bins=32)
    ph = W.homogeneous((8, 8, 8), 0.5, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    try:
        grouped = W.Source(W.PHOTON, W.BEAM_PENCIL, center_cm=(2.0, 2.0), spectrum_edges=edges,
                           spectrum_weights=w, energy_grouping=W.ENERGY_GROUPED)
        plain = W.Source(W.PHOTON, W.BEAM_PENCIL, center_cm=(2.0, 2.0), spectrum_edges=edges,
                         spectrum_weights=w)
        pg = ctx.plan_open(pid, grouped, 1, 16)
        pp = ctx.plan_open(pid, plain, 1, 16)
        ctx.set_launch(flags=g.LAUNCH_KERMA)
        with pytest.raises(g.GpumcdError) as e:
            ctx.run([pg], [64])
        assert e.value.status == g.ERR_INVALID_ARG
        ctx.run([pp], [64])
        ctx.set_launch(flags=0)
        ctx.run([pg], [64])
        assert ctx.plan_result(pg, 0.5)["histories"] == 64
        ctx.plan_close(pg)
        ctx.plan_close(pp)
    finally:
        ctx.set_launch(flags=0)
        ctx.destroy_phantom(pid)


def test_grouped_spectrum_claims_past_2_to_24_histories(ctx):
    """The claim order is sorted per launch from the launch's own histories, so
    it holds at any history index: after 2^24 histories, one more run of a
    grouped spectrum still equals the ungrouped run on the same kernel."""
    edges, w = W.synthetic_6mv_spectrum(n_bins=64)
    ph = W.homogeneous((8, 8, 8), 0.5, W.MAT_LUNG, 0.05)
    kw = dict(center_cm=(2.0, 2.0), spectrum_edges=edges, spectrum_weights=w)
    a = _phsp_kernel_runs(ctx, ph, W.Source(W.PHOTON, W.BEAM_PENCIL, energy_grouping=W.ENERGY_GROUPED, **kw), 5,
                          [1 << 24, 70_001])
    b = _phsp_kernel_runs(ctx, ph, W.Source(W.PHOTON, W.BEAM_PENCIL, **kw), 5, [(1 << 24) + 70_001])
    assert a[2]["histories"] == (1 << 24) + 70_001 and ledger_exact(a[2])
    assert np.array_equal(a[0], b[0]) and a[2]["e_incident"] == b[2]["e_incident"]

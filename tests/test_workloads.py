"""Checks of the seeded input recipes (workloads/)."""
import numpy as np
import pytest

import workloads as W


def test_materials_fractions():
    for m in W.MATERIALS_PAPER:
        assert sum(m.w) == pytest.approx(1.0, abs=1e-12)
        assert len(m.Z) <= W.MAX_ELEMENTS
    assert W.WATER.w[0] == pytest.approx(0.1119, abs=2e-4)


def test_paper_geometries():
    """GPUMCD §III.A: the lung box (electrons 4 cm from 3 cm depth, photons
    6.5 cm from 5.5 cm; 4.5 cm wide, on the axis) and the tissue / lung /
    bone slabs (2/2/2 cm and 3/2/7 cm), on 128^3 at 0.25 cm."""
    assert W.MATERIALS_PAPER[:3] == W.MATERIALS and W.MATERIALS_PAPER[W.MAT_TISSUE].name == "tissue"
    for particle, (z0, z1) in ((W.ELECTRON, (12, 28)), (W.PHOTON, (22, 48))):
        ph = W.geom2(particle).phantom
        col = ph.mat[:, 64, 64]
        assert (col[z0:z1] == W.MAT_LUNG).all() and (col[:z0] == W.MAT_WATER).all()
        assert (col[z1:] == W.MAT_WATER).all()
        row = ph.mat[(z0 + z1) // 2, 64, :]
        assert int((row == W.MAT_LUNG).sum()) == 18  # 4.5 cm
        assert np.allclose(ph.rho[ph.mat == W.MAT_LUNG], 0.26)
    for particle, cuts in ((W.ELECTRON, (8, 16, 24)), (W.PHOTON, (12, 20, 48))):
        ph = W.geom3(particle).phantom
        col = ph.mat[:, 10, 100]
        a, b, c = cuts
        assert (col[:a] == W.MAT_TISSUE).all() and (col[a:b] == W.MAT_LUNG).all()
        assert (col[b:c] == W.MAT_BONE).all() and (col[c:] == W.MAT_TISSUE).all()
        assert np.allclose(ph.rho[:, 10, 100][b:c], 1.85)


def test_hu_calibration_and_thresholds():
    """The HU -> density curve passes through its points, is monotone, and the
    material follows the HU thresholds."""
    hu = np.array([-1000.0, -740.0, -400.0, -1.0, 0.0, 249.0, 250.0, 1400.0, 3000.0, 5000.0]).reshape(1, 1, -1)
    ph = W.hu_to_phantom(hu, 0.5)
    rho, mat = ph.rho.ravel(), ph.mat.ravel()
    assert rho[0] == np.float32(0.0012) and rho[1] == np.float32(0.26) and rho[4] == np.float32(1.0)
    assert rho[7] == np.float32(1.85) and rho[8] == np.float32(2.8) and rho[9] == np.float32(2.8)
    assert np.all(np.diff(rho) >= 0)
    assert list(mat) == [W.MAT_LUNG, W.MAT_LUNG, W.MAT_TISSUE, W.MAT_TISSUE, W.MAT_TISSUE, W.MAT_TISSUE,
                         W.MAT_BONE, W.MAT_BONE, W.MAT_BONE, W.MAT_BONE]


def test_synthetic_ct_is_seeded_and_thorax_like():
    a = W.synthetic_ct_hu((40, 8, 40), 0.5, 6)
    b = W.synthetic_ct_hu((40, 8, 40), 0.5, 6)
    c = W.synthetic_ct_hu((40, 8, 40), 0.5, 7)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    ph = W.synthetic_ct(W.PHOTON, dims=(64, 16, 64), voxel_cm=0.5).phantom
    frac = {m: float((ph.mat == m).mean()) for m in (W.MAT_LUNG, W.MAT_BONE, W.MAT_TISSUE)}
    assert 0.3 < frac[W.MAT_TISSUE] < 0.5 and 0.005 < frac[W.MAT_BONE] < 0.05
    assert ph.rho.min() == np.float32(0.0012) and 1.6 < ph.rho.max() < 1.9
    # the beam axis crosses tissue, the sternum and a lung-free mediastinum
    col = ph.mat[:, 8, 32]
    assert W.MAT_BONE in col and W.MAT_TISSUE in col


def test_config3_slabs():
    pl = W.config3(n=256, voxel_cm=0.2)
    ph = pl.phantom
    col = ph.mat[:, 0, 0]
    rho = ph.rho[:, 0, 0]
    # 3 cm water, 2 cm bone, 6 cm lung, rest water at 0.2 cm voxels
    assert (col[:15] == W.MAT_WATER).all() and (rho[:15] == 1.0).all()
    assert (col[15:25] == W.MAT_BONE).all() and np.allclose(rho[15:25], 1.85)
    assert (col[25:55] == W.MAT_LUNG).all() and np.allclose(rho[25:55], 0.26)
    assert (col[55:] == W.MAT_WATER).all()
    e, w = pl.source.spectrum_edges, pl.source.spectrum_weights
    assert e[0] == pytest.approx(0.1) and e[-1] == pytest.approx(6.0)
    assert len(w) == 256 and w.sum() == pytest.approx(1.0) and (w >= 0).all()


def test_spectrum_is_seeded():
    a = W.synthetic_6mv_spectrum(seed=3)[1]
    b = W.synthetic_6mv_spectrum(seed=3)[1]
    c = W.synthetic_6mv_spectrum(seed=4)[1]
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_plan_distribution_ranges():
    specs = W.config4()
    assert len(specs) == 64
    for s in specs:
        assert 64 <= s.n <= 256
        assert 0.2 <= s.voxel_cm <= 0.5
        assert 6.0 <= s.energy <= 18.0
        assert 2.0 <= s.field_cm <= 15.0
        assert 1e5 <= s.n_histories <= 1e7
    assert {s.particle for s in specs} == {W.PHOTON, W.ELECTRON}


def test_smoothed_noise_phantom():
    spec = W.config4()[0]
    ph = W.smoothed_noise(48, 0.4, np.random.default_rng(spec.phantom_seed))
    assert ph.rho.min() == pytest.approx(0.2, abs=1e-6)
    assert ph.rho.max() == pytest.approx(2.0, abs=1e-6)
    assert (ph.mat[ph.rho < 0.6] == W.MAT_LUNG).all()
    assert (ph.mat[ph.rho > 1.4] == W.MAT_BONE).all()


def test_config5_arrivals():
    reqs = W.config5(count=50, rate_per_s=20.0)
    t = np.array([r.arrival_s for r in reqs])
    assert (np.diff(t) > 0).all()


def test_point_source_phase_space_recipe():
    """Seeded records on the entry face, inside the field, unit directions
    pointing away from the source point, energies in range."""
    ph = W.homogeneous((40, 40, 10), 0.5, W.MAT_WATER, 1.0)
    a = W.point_source_phase_space(W.PHOTON, ph, 500, seed=3, field_cm=8.0, e_lo=1.0, e_hi=12.0)
    b = W.point_source_phase_space(W.PHOTON, ph, 500, seed=3, field_cm=8.0, e_lo=1.0, e_hi=12.0)
    ps = a.phase_space
    assert a.beam == W.BEAM_PHASE_SPACE and ps.shape == (500, 7) and np.array_equal(ps, b.phase_space)
    assert np.all(ps[:, 2] == 0.0)
    assert np.all(np.abs(ps[:, 0] - 10.0) <= 4.0) and np.all(np.abs(ps[:, 1] - 10.0) <= 4.0)
    assert np.allclose(np.linalg.norm(ps[:, 3:6], axis=1), 1.0)
    # each direction lies on the ray from the source point 30 cm above the field centre
    src = np.array([10.0, 10.0, -30.0])
    d = ps[:, 0:3] - src
    assert np.allclose(d / np.linalg.norm(d, axis=1, keepdims=True), ps[:, 3:6])
    assert ps[:, 6].min() >= 1.0 and ps[:, 6].max() <= 12.0 and a.max_energy == ps[:, 6].max()


def test_polyenergetic_phase_space_recipe():
    """Spectrum draws stay inside the bins and follow the weights; photon
    records span the 6 MV-like spectrum, electron records 1-15 MeV; both are
    seeded."""
    edges, w = W.synthetic_6mv_spectrum()
    e = W.draw_spectrum(edges, w, 200_000, seed=4)
    assert e.min() >= edges[0] and e.max() <= edges[-1]
    h, _ = np.histogram(e, bins=edges)
    want = w * len(e)
    big = want > 400
    assert np.all(np.abs(h[big] - want[big]) <= 5 * np.sqrt(want[big]))
    ph = W.homogeneous((40, 40, 10), 0.5, W.MAT_WATER, 1.0)
    for particle, lo, hi in ((W.PHOTON, 0.1, 6.0), (W.ELECTRON, 1.0, 15.0)):
        a = W.polyenergetic_phase_space(particle, ph, 3000, seed=8)
        b = W.polyenergetic_phase_space(particle, ph, 3000, seed=8)
        assert np.array_equal(a.phase_space, b.phase_space)
        assert a.energy_grouping == W.ENERGY_UNGROUPED
        assert lo <= a.phase_space[:, 6].min() and a.phase_space[:, 6].max() <= hi
        assert a.phase_space[:, 6].max() - a.phase_space[:, 6].min() > 0.8 * (hi - lo) - 1.0

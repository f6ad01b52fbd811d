"""Pins for the oracle's photon physics and Woodcock tracking (GPUMCD §II.A).

Each check compares the oracle with something other than itself: textbook
values, a numerical quadrature of the differential cross-section, an analytic
density (chi-square), or an exact attenuation law.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import workloads as W
from tests._stats import chi2_pvalue, within_sigma

RE = 2.8179403262e-13
MC2 = 0.51099895
SIGMA_T = 8.0 * math.pi / 3.0 * RE * RE
P = W.DEFAULT_PHYSICS


def test_klein_nishina_textbook_values():
    L = oracle.lib()
    # sigma_KN at k = 1 is 2 pi re^2 x 0.57430 = 0.2865 barn
    assert L.om_sigma_kn(1.0) / 1e-24 == pytest.approx(0.28654, rel=2e-4)
    # Thomson limit: sigma -> (8 pi / 3) re^2 (1 - 2k + ...) as k -> 0
    for k in (1e-3, 1e-4):
        assert L.om_sigma_kn(k) / SIGMA_T == pytest.approx(1.0 - 2.0 * k, abs=1e-5)


@pytest.mark.parametrize("k", [0.02, 0.3, 1.0, 5.0, 39.0])
def test_klein_nishina_total_equals_quadrature(k):
    L = oracle.lib()
    val, _ = integrate.quad(lambda c: L.om_kn_dsigma_domega(k, c), -1.0, 1.0, epsabs=0,
                            epsrel=1e-13, limit=200, points=[1.0 - 1.0 / k] if k > 0.5 else None)
    assert 2.0 * math.pi * val == pytest.approx(L.om_sigma_kn(k), rel=1e-10)


def kn_density(k):
    def f(c):
        r = 1.0 / (1.0 + k * (1.0 - c))
        return r * r * (r + 1.0 / r - (1.0 - c * c))
    return f


@pytest.mark.parametrize("k", [0.1, 1.0, 10.0, 30.0])
def test_klein_nishina_sampler_chi2(k):
    cos, eps = oracle.sample("kn", 200_000, 11, k)
    # the sampled energy fraction is the Compton relation of the sampled angle
    assert np.allclose(eps, 1.0 / (1.0 + k * (1.0 - cos)), rtol=1e-12)
    grid = 1.0 - np.geomspace(2.0, 1e-7, 20001)
    grid = np.concatenate([grid, [1.0]])
    assert chi2_pvalue(cos, kn_density(k), grid) > 0.01


def test_water_compton_attenuation_textbook():
    """Water's Compton mass attenuation coefficient at 1 MeV, where binding
    effects are negligible and Compton scattering is the whole of the
    attenuation: the tabulated 0.0707 cm^2/g.  It ties the electron density
    (electrons per gram) to the Klein-Nishina cross-section."""
    assert oracle.xs("mu_compton", W.WATER, 1.0) == pytest.approx(0.0707, rel=5e-3)


def test_photoelectric_scaling():
    """Born K-shell form: sigma ~ Z^5 k^-7/2 per atom."""
    m = W.WATER
    r = oracle.xs("mu_photo", m, 0.02) / oracle.xs("mu_photo", m, 0.04)
    assert r == pytest.approx(2.0 ** 3.5, rel=1e-12)
    # water at 30 keV: 4 sqrt2 alpha^4 Z^5 sigma_T k^-3.5 summed over O and H
    alpha = 1 / 137.035999084
    k = 0.03 / MC2
    expect = sum(6.02214076e23 * w / A * 4 * math.sqrt(2) * alpha ** 4 * Z ** 5 * SIGMA_T * k ** -3.5
                 for Z, A, w in zip(m.Z, m.A, m.w))
    assert oracle.xs("mu_photo", m, 0.03) == pytest.approx(expect, rel=1e-12)
    assert 0.1 < expect < 0.4  # tabulated water photoelectric at 30 keV is ~0.15 cm^2/g


def _sauter_k_shell(Z: int, k: float) -> float:
    """Sauter's relativistic Born cross-section per atom for the K-shell photo
    effect, binding neglected in the final state (Heitler, The Quantum Theory of
    Radiation, section 21): (3/2) sigma_T Z^5 alpha^4 k^-5 (g^2 - 1)^(3/2)
    [4/3 + g (g - 2) / (g + 1) (1 - ln(g + sqrt(g^2 - 1)) / (g sqrt(g^2 - 1)))],
    with k = E / mc^2 and g = k + 1 the photo-electron's total energy in mc^2."""
    alpha = 1 / 137.035999084
    g = k + 1.0
    s = math.sqrt(k * (k + 2.0))  # sqrt(g^2 - 1), without cancellation
    bracket = 4.0 / 3.0 + g * (g - 2.0) / (g + 1.0) * (1.0 - math.asinh(s) / (g * s))
    return 1.5 * SIGMA_T * Z ** 5 * alpha ** 4 * k ** -5 * s ** 3 * bracket


def test_photoelectric_magnitude_is_the_low_energy_limit_of_sauter():
    """The oracle's K-shell photoelectric cross-section (the non-relativistic
    Born form) is the k -> 0 limit of Sauter's relativistic formula, an
    independent published expression.  Their ratio is 1 + k/4 + O(k^2), so a
    wrong constant (a dropped sqrt 2, alpha^3, r_e^2 for sigma_T) or a wrong
    power of Z fails it.  The transcription of Sauter's formula is checked by
    its own high-energy limit, (3/2) sigma_T Z^5 alpha^4 / k."""
    alpha = 1 / 137.035999084
    for symbol in ("O", "Ca"):
        el = W.Material("pure", ((symbol, 1.0),), 95.0, 1.0)
        Z, A = el.Z[0], el.A[0]
        for k in (1e-5, 1e-4, 1e-3):
            per_atom = oracle.xs("mu_photo", el, k * MC2) * A / 6.02214076e23
            ratio = per_atom / _sauter_k_shell(Z, k)
            assert ratio == pytest.approx(1.0 / (1.0 + k / 4.0), rel=5.0 * k * k + 1e-12), (Z, k, ratio)
        k = 1e7
        assert _sauter_k_shell(Z, k) * k / (1.5 * SIGMA_T * Z ** 5 * alpha ** 4) == pytest.approx(1.0, rel=1e-5)


def test_pair_threshold_and_asymptote():
    for E in (0.5, 1.0, 2 * MC2):
        assert oracle.xs("mu_pair", W.WATER, E) == 0.0
    assert oracle.xs("mu_pair", W.WATER, 2 * MC2 + 0.01) > 0.0
    # above threshold the energy dependence is exactly (1 - 2mc^2/E)^3
    a = oracle.xs("mu_pair", W.BONE, 3.0) / (1 - 2 * MC2 / 3.0) ** 3
    b = oracle.xs("mu_pair", W.BONE, 17.0) / (1 - 2 * MC2 / 17.0) ** 3
    assert a == pytest.approx(b, rel=1e-13)


def sauter_density(T):
    g = T / MC2 + 1.0
    beta = math.sqrt(1 - 1 / g ** 2)

    def f(c):
        s2 = 1.0 - c * c
        x = 1.0 - beta * c
        return s2 / x ** 4 * (1.0 + 0.5 * g * (g - 1.0) * (g - 2.0) * x)
    return f


@pytest.mark.parametrize("T", [0.02, 0.3, 1.5, 5.0])
def test_sauter_sampler_chi2(T):
    cos = oracle.sample("sauter", 200_000, 12, T)
    assert np.all((cos >= -1.0) & (cos <= 1.0))
    grid = np.concatenate([[-1.0], 1.0 - np.geomspace(2.0, 1e-9, 30000)[1:], [1.0]])
    assert chi2_pvalue(cos, sauter_density(T), grid) > 0.01


def test_spectrum_sampler_chi2():
    edges, w = W.synthetic_6mv_spectrum(seed=3)
    e = oracle.sample("spectrum", 1_000_000, 13, edges, w)
    counts, _ = np.histogram(e, bins=edges)
    from scipy import stats
    assert stats.chisquare(counts, w * len(e) / w.sum()).pvalue > 0.01
    # uniform inside a bin
    i = int(np.argmax(w))
    inside = e[(e >= edges[i]) & (e < edges[i + 1])]
    frac = (inside - edges[i]) / (edges[i + 1] - edges[i])
    assert stats.kstest(frac, "uniform").pvalue > 0.01


def _transmission(ph, E, depths, n=200_000, seed=21):
    src = W.pencil(W.PHOTON, E, ph.extent_cm[0] / 2, ph.extent_cm[1] / 2)
    z, nf = oracle.first_interaction_z(W.MATERIALS, P, ph, src, n, seed)
    out = []
    for x in depths:
        p = float(np.mean(z > x))
        out.append((p, math.sqrt(max(p * (1 - p), 1e-12) / n)))
    return out, nf


@pytest.mark.parametrize("E", [0.05, 1.25, 15.0])
def test_narrow_beam_transmission_water(E):
    """Uncollided fraction at depth x is exp(-mu x) (distance equation, §II.A)."""
    ph = W.homogeneous((4, 4, 60), 0.5, W.MAT_WATER, 1.0)
    mu = oracle.xs("mu_total", W.WATER, E)
    depths = [0.5, 3.0, 10.0, 25.0]
    res, nf = _transmission(ph, E, depths)
    assert nf == 0  # the majorant equals mu in a homogeneous phantom
    for (p, s), x in zip(res, depths):
        assert within_sigma(p, math.exp(-mu * x), s), (x, p, math.exp(-mu * x), s)


@pytest.mark.parametrize("E", [0.08, 2.0])
def test_narrow_beam_transmission_slabs_woodcock(E):
    """Through water/bone/lung/water slabs the uncollided fraction is
    exp(-sum mu_i x_i): Woodcock tracking is exact in heterogeneous media."""
    slabs = [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85), (6.0, W.MAT_LUNG, 0.26),
             (1e9, W.MAT_WATER, 1.0)]
    ph = W.z_slabs((4, 4, 60), 0.5, slabs)
    mw = oracle.xs("mu_total", W.WATER, E)
    mb = 1.85 * oracle.xs("mu_total", W.BONE, E)
    ml = 0.26 * oracle.xs("mu_total", W.LUNG, E)

    def optical(x):
        t = min(x, 3.0) * mw
        t += max(0.0, min(x, 5.0) - 3.0) * mb
        t += max(0.0, min(x, 11.0) - 5.0) * ml
        t += max(0.0, x - 11.0) * mw
        return t
    depths = [2.0, 4.0, 8.0, 14.0]
    res, nf = _transmission(ph, E, depths)
    assert nf > 0  # water and lung voxels see fictitious events
    for (p, s), x in zip(res, depths):
        assert within_sigma(p, math.exp(-optical(x)), s), (x, p, math.exp(-optical(x)), s)


def _kn_mean_eps(k):
    f = kn_density(k)
    num, _ = integrate.quad(lambda c: f(c) / (1 + k * (1 - c)), -1, 1, epsrel=1e-12, limit=200)
    den, _ = integrate.quad(f, -1, 1, epsrel=1e-12, limit=200)
    return num / den


@pytest.mark.parametrize("E", [0.2, 2.0, 12.0])
def test_first_collision_kerma_depth_dose(E):
    """Brute force on a water column: with the first real interaction ending the
    photon and electrons deposited on the spot, the energy left in slab
    [z0, z1] is N e^{-mu z0}(1 - e^{-mu dz}) times the mean energy transferred,
    (mu_C E (1 - <k'/k>) + mu_pe E + mu_pp (E - 2mc^2)) / mu."""
    n = 60_000
    ph = W.homogeneous((1, 1, 40), 0.5, W.MAT_WATER, 1.0)
    ph = W.Phantom(ph.dims, (50.0, 50.0, 0.5), ph.mat, ph.rho)
    src = W.pencil(W.PHOTON, E, 25.0, 25.0)
    res = oracle.simulate(W.MATERIALS, P, ph, src, n, 5,
                          flags=oracle.FLAG_KERMA | oracle.FLAG_FIRST_COLLISION)
    st = res.stats
    assert st["e_deposited"] + st["e_escaped"] + st["e_rest"] == pytest.approx(
        st["e_incident"], rel=1e-12)
    muC = oracle.xs("mu_compton", W.WATER, E)
    mupe = oracle.xs("mu_photo", W.WATER, E)
    mupp = oracle.xs("mu_pair", W.WATER, E)
    mu = muC + mupe + mupp
    etr = (muC * E * (1 - _kn_mean_eps(E / MC2)) + mupe * E + mupp * (E - 2 * MC2)) / mu
    z = np.arange(41) * 0.5
    expect = n * np.exp(-mu * z[:-1]) * (1 - np.exp(-mu * 0.5)) * etr
    sig = np.sqrt(np.maximum(res.sum_e2 - res.sum_e ** 2 / n, 0))
    ok = np.abs(res.sum_e - expect) <= 3 * sig + 1e-9
    assert ok.mean() >= 0.95, np.c_[res.sum_e, expect, sig][~ok]
    assert res.sum_e.sum() == pytest.approx(expect.sum(), rel=5 * math.sqrt(
        max((sig ** 2).sum(), 1e-30)) / expect.sum() + 1e-9)


def test_woodcock_invariance_far_dense_voxel():
    """Raising the majorant with one far-away dense voxel changes nothing but
    the number of fictitious events (§II.A: Woodcock is not an approximation)."""
    from tests._stats import three_sigma_pass_rate
    base = W.homogeneous((16, 16, 24), 0.5, W.MAT_WATER, 1.0)
    dense = W.homogeneous((16, 16, 24), 0.5, W.MAT_WATER, 1.0)
    dense.mat[23, 0, 0] = W.MAT_BONE
    dense.rho[23, 0, 0] = 2.0
    src = W.pencil(W.PHOTON, 1.25, 4.0, 4.0)
    n = 30_000
    a = oracle.simulate(W.MATERIALS, P, base, src, n, 7)
    b = oracle.simulate(W.MATERIALS, P, dense, src, n, 8)
    assert a.stats["n_photon_fict"] == 0 and b.stats["n_photon_fict"] > 0
    da, sa = a.dose_gy(base), a.sigma_gy(base)
    db, sb = b.dose_gy(dense), b.sigma_gy(dense)
    mask = da > 0.1 * da.max()
    mask[23 * 16 * 16] = False  # the dense voxel itself
    assert three_sigma_pass_rate(da, sa, db, sb, mask) >= 0.98


def test_phase_space_source_equals_the_beam_it_lists():
    """A phase-space source (the paper's outlook, §V) whose every record is the
    pencil beam's primary - same point, +z, same energy - gives the pencil
    run's tallies exactly: record h mod n starts history h, and neither form
    draws a random number for the primary."""
    ph = W.homogeneous((12, 12, 20), 0.5, W.MAT_WATER, 1.0)
    pen = W.pencil(W.PHOTON, 3.0, 3.0, 3.0)
    rec = np.array([[3.0, 3.0, 0.0, 0.0, 0.0, 2.0, 3.0]])  # direction need not be unit length
    phs = W.Source(W.PHOTON, W.BEAM_PHASE_SPACE, phase_space=np.repeat(rec, 5, axis=0))
    a = oracle.simulate(W.MATERIALS, P, ph, pen, 2000, 9)
    b = oracle.simulate(W.MATERIALS, P, ph, phs, 2000, 9)
    assert np.array_equal(a.sum_e, b.sum_e) and np.array_equal(a.sum_e2, b.sum_e2)


def test_phase_space_records_cycle_and_conserve_energy():
    """History h takes record h mod n: the incident energy of N histories is the
    sum of the records' energies taken in turn, and the ledger closes."""
    ph = W.homogeneous((16, 16, 16), 0.5, W.MAT_WATER, 1.0)
    src = W.point_source_phase_space(W.ELECTRON, ph, 7, seed=3, field_cm=4.0)
    n = 50
    r = oracle.simulate(W.MATERIALS, P, ph, src, n, 4)
    want = sum(src.phase_space[h % 7, 6] for h in range(n))
    st = r.stats
    assert st["e_incident"] == pytest.approx(want, rel=1e-12)
    assert st["e_deposited"] + st["e_escaped"] + st["e_rest"] == pytest.approx(st["e_incident"], rel=1e-9)


def test_phase_space_grouped_by_energy_takes_the_records_as_listed():
    """Energy grouping (§IV's grouping of similar energies) of a phase space is
    a schedule: the GPU claims a launch's histories in decreasing order of
    their record's energy, and history h still starts as record h mod n of the
    list as given.  So over a ragged number of histories (a partial last
    cycle, where a list reordered by energy would start other records) the
    incident energy is the listed records' sum taken in turn, and the tallies
    equal the ungrouped ones bit for bit."""
    ph = W.homogeneous((14, 14, 16), 0.5, W.MAT_WATER, 1.0)
    src = W.point_source_phase_space(W.ELECTRON, ph, 9, seed=5, field_cm=4.0)
    n = 67
    grouped = W.Source(W.ELECTRON, W.BEAM_PHASE_SPACE, phase_space=src.phase_space,
                       energy_grouping=W.ENERGY_GROUPED)
    a = oracle.simulate(W.MATERIALS, P, ph, grouped, n, 6)
    b = oracle.simulate(W.MATERIALS, P, ph, src, n, 6)
    want = sum(src.phase_space[h % 9, 6] for h in range(n))
    assert a.stats["e_incident"] == pytest.approx(want, rel=1e-12)
    rows = sorted(range(9), key=lambda i: -src.phase_space[i, 6])
    assert abs(sum(src.phase_space[rows[h % 9], 6] for h in range(n)) - want) > 1.0  # a sorted list differs
    assert np.array_equal(a.sum_e, b.sum_e) and np.array_equal(a.sum_e2, b.sum_e2)


def _strata_deviation(e, edges, w):
    """Largest |#(E < edge_i) - n * CDF(edge_i)| over the spectrum's edges."""
    cdf = np.concatenate([[0.0], np.cumsum(w) / np.sum(w)])
    counts = np.searchsorted(np.sort(e), edges, side="left")
    return float(np.max(np.abs(counts - len(e) * cdf)))


def test_grouped_spectrum_draws_what_an_ungrouped_one_draws():
    """Energy grouping (§IV's grouping of similar energies) of a spectrum is a
    schedule: the GPU claims a launch's histories in decreasing order of their
    energy, and each history draws its energy as it would ungrouped.  So the
    oracle's grouped and ungrouped spectra give the same energies and the same
    tallies; a monoenergetic beam is unchanged."""
    edges, w = W.synthetic_6mv_spectrum(n_bins=64)
    grouped = W.Source(W.PHOTON, W.BEAM_PENCIL, center_cm=(1.0, 1.0), spectrum_edges=edges,
                       spectrum_weights=w, energy_grouping=W.ENERGY_GROUPED)
    plain = W.Source(W.PHOTON, W.BEAM_PENCIL, center_cm=(1.0, 1.0), spectrum_edges=edges,
                     spectrum_weights=w)
    a = oracle.primary_energies(grouped, 70_000, 72_000, seed=12)
    b = oracle.primary_energies(plain, 70_000, 72_000, seed=12)
    assert np.array_equal(a, b)
    assert _strata_deviation(a, edges, w) > 3.0  # iid draws, not strata
    ph = W.homogeneous((8, 8, 16), 0.5, W.MAT_WATER, 1.0)
    ra = oracle.simulate(W.MATERIALS, P, ph, grouped, 500, 3)
    rb = oracle.simulate(W.MATERIALS, P, ph, plain, 500, 3)
    assert np.array_equal(ra.sum_e, rb.sum_e)
    mono = W.Source(W.PHOTON, W.BEAM_PENCIL, energy=2.0, energy_grouping=W.ENERGY_GROUPED)
    assert np.all(oracle.primary_energies(mono, 0, 50, seed=1) == 2.0)

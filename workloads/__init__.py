"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and bench.py.

This module holds input data and input recipes only: element data, material
compositions, voxel phantoms, beam sources and the photon spectrum weights.  It
contains none of the transport method's arithmetic (no cross-sections, stopping
powers or samplers): both the oracle and the CUDA library derive everything they
compute from these inputs on their own.

Workloads follow the phantoms and beams of GPUMCD §III (slab geometries, 15 MeV
parallel beams, §II.D: 1M electrons / 4M photons) scaled to the sizes listed in
``CONFIGS`` below.  Voxel order everywhere is x fastest, then y, then z, and the
beam enters through the z = 0 face travelling along +z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Element data (Z, standard atomic weight in g/mol).
# ---------------------------------------------------------------------------
ELEMENTS = {
    "H": (1, 1.008),
    "C": (6, 12.011),
    "N": (7, 14.007),
    "O": (8, 15.999),
    "Na": (11, 22.990),
    "Mg": (12, 24.305),
    "P": (15, 30.974),
    "S": (16, 32.06),
    "Ca": (20, 40.078),
}

MAX_ELEMENTS = 16


@dataclasses.dataclass(frozen=True)
class Material:
    """A homogeneous material: element mass fractions and mean excitation energy."""

    name: str
    elements: Tuple[Tuple[str, float], ...]  # (symbol, mass fraction)
    I_eV: float
    nominal_density: float

    @property
    def Z(self) -> List[int]:
        return [ELEMENTS[s][0] for s, _ in self.elements]

    @property
    def A(self) -> List[float]:
        return [ELEMENTS[s][1] for s, _ in self.elements]

    @property
    def w(self) -> List[float]:
        tot = sum(f for _, f in self.elements)
        return [f / tot for _, f in self.elements]


def _water_fractions() -> Tuple[Tuple[str, float], ...]:
    aH, aO = ELEMENTS["H"][1], ELEMENTS["O"][1]
    m = 2 * aH + aO
    return (("H", 2 * aH / m), ("O", aO / m))


WATER = Material("water", _water_fractions(), 75.0, 1.0)
# Lung: water composition at lung density (the density lives in the phantom).
LUNG = Material("lung", _water_fractions(), 75.0, 0.26)
# Cortical bone, ICRU-44-like mass fractions.
BONE = Material(
    "bone",
    (("H", 0.034), ("C", 0.155), ("N", 0.042), ("O", 0.435), ("Na", 0.001),
     ("Mg", 0.002), ("P", 0.103), ("S", 0.003), ("Ca", 0.225)),
    106.4,
    1.85,
)

MATERIALS: Tuple[Material, ...] = (WATER, LUNG, BONE)
MAT_WATER, MAT_LUNG, MAT_BONE = 0, 1, 2
# Soft tissue for the paper's third geometry (GPUMCD §III.A), which names the
# material but not its data: the ICRU four-component soft tissue (mass
# fractions H 0.101, C 0.111, N 0.026, O 0.762; I = 74.9 eV; 1.0 g/cm^3).
TISSUE = Material("tissue", (("H", 0.101), ("C", 0.111), ("N", 0.026), ("O", 0.762)), 74.9, 1.0)
# The material set of the paper's geometries: the three above plus tissue.
MATERIALS_PAPER: Tuple[Material, ...] = (WATER, LUNG, BONE, TISSUE)
MAT_TISSUE = 3


@dataclasses.dataclass(frozen=True)
class Physics:
    """Transport cut-offs and thresholds (MeV) and the electron step controls.

    p_cut  : photon cut-off (GPUMCD §II.A, P_cut; 0.01 MeV as in §II.D)
    e_abs  : electron kinetic-energy cut-off (absorbed below it)
    t_c    : Moller knock-on threshold (hard inelastic collisions above it)
    k_c    : bremsstrahlung photon threshold (hard radiative events above it)
    estepe : largest fractional CSDA energy loss per step (the e_s-max bound)
    e_max  : top of the energy range covered by the tables
    nudge_cm : distance added to the voxel-boundary distance so a step that is
               limited by it always ends past the boundary
    """

    p_cut: float = 0.01
    e_abs: float = 0.2
    t_c: float = 0.2
    k_c: float = 0.01
    estepe: float = 0.25
    e_max: float = 20.0
    nudge_cm: float = 1e-4


DEFAULT_PHYSICS = Physics()


@dataclasses.dataclass
class Phantom:
    dims: Tuple[int, int, int]
    voxel_cm: Tuple[float, float, float]
    mat: np.ndarray  # uint8, shape (nz, ny, nx) (x fastest in memory)
    rho: np.ndarray  # float32, same shape, g/cm^3

    @property
    def nvox(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz

    @property
    def extent_cm(self) -> Tuple[float, float, float]:
        return tuple(n * d for n, d in zip(self.dims, self.voxel_cm))  # type: ignore

    def nbytes(self) -> int:
        return self.mat.nbytes + self.rho.nbytes


PHOTON, ELECTRON = 0, 1
BEAM_PENCIL, BEAM_SQUARE, BEAM_PHASE_SPACE = 0, 1, 2
ENERGY_UNGROUPED, ENERGY_GROUPED = 0, 1


@dataclasses.dataclass
class Source:
    particle: int  # PHOTON or ELECTRON
    beam: int  # BEAM_PENCIL, BEAM_SQUARE or BEAM_PHASE_SPACE
    energy: float = 0.0  # MeV, used when spectrum is None
    center_cm: Tuple[float, float] = (0.0, 0.0)  # beam centre on the z = 0 face
    field_cm: float = 0.0  # side of the square field
    spectrum_edges: Optional[np.ndarray] = None  # float64, n+1 bin edges (MeV)
    spectrum_weights: Optional[np.ndarray] = None  # float64, n bin weights
    # BEAM_PHASE_SPACE: records (n, 7) = x, y, z (cm), ux, uy, uz, E (MeV), all of
    # `particle`; history h starts as record h mod n
    phase_space: Optional[np.ndarray] = None
    # ENERGY_GROUPED (spectra and phase spaces): each launch claims its
    # histories in decreasing order of their primary's energy, so that the
    # histories started together have nearby energies (§IV); every history
    # starts as it would ungrouped
    energy_grouping: int = ENERGY_UNGROUPED

    @property
    def max_energy(self) -> float:
        if self.phase_space is not None:
            return float(np.max(self.phase_space[:, 6]))
        if self.spectrum_edges is not None:
            return float(self.spectrum_edges[-1])
        return self.energy


@dataclasses.dataclass
class Plan:
    """One dose calculation: a phantom, a beam, a history count and a seed."""

    name: str
    phantom: Phantom
    source: Source
    n_histories: int
    seed: int


# ---------------------------------------------------------------------------
# Phantom recipes
# ---------------------------------------------------------------------------
def homogeneous(n: Sequence[int], voxel_cm: float, mat_id: int, density: float) -> Phantom:
    nx, ny, nz = n
    mat = np.full((nz, ny, nx), mat_id, dtype=np.uint8)
    rho = np.full((nz, ny, nx), density, dtype=np.float32)
    return Phantom((nx, ny, nz), (voxel_cm,) * 3, mat, rho)


def z_slabs(n: Sequence[int], voxel_cm: float,
            slabs: Sequence[Tuple[float, int, float]]) -> Phantom:
    """Slabs stacked along z: each entry (thickness_cm, material id, density).

    The last slab extends to the end of the grid whatever its thickness.
    """
    nx, ny, nz = n
    mat = np.zeros((nz, ny, nx), dtype=np.uint8)
    rho = np.zeros((nz, ny, nx), dtype=np.float32)
    z0 = 0
    for i, (thick, m, d) in enumerate(slabs):
        z1 = nz if i == len(slabs) - 1 else min(nz, z0 + int(round(thick / voxel_cm)))
        mat[z0:z1] = m
        rho[z0:z1] = d
        z0 = z1
    return Phantom((nx, ny, nz), (voxel_cm,) * 3, mat, rho)


def box_in_water(n: Sequence[int], voxel_cm: float, box_lo_cm: Sequence[float],
                 box_hi_cm: Sequence[float], mat_id: int, density: float) -> Phantom:
    """Water with an axis-aligned box of another material (GPUMCD §III.A Geom2)."""
    ph = homogeneous(n, voxel_cm, MAT_WATER, 1.0)
    lo = [int(round(v / voxel_cm)) for v in box_lo_cm]
    hi = [int(round(v / voxel_cm)) for v in box_hi_cm]
    ph.mat[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = mat_id
    ph.rho[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = density
    return ph


def smoothed_noise(n: int, voxel_cm: float, rng: np.random.Generator,
                   sigma_cm: float = 2.0, rho_lo: float = 0.2, rho_hi: float = 2.0,
                   lung_below: float = 0.6, bone_above: float = 1.4) -> Phantom:
    """Seeded heterogeneous phantom: Gaussian white noise smoothed by a Gaussian
    kernel of ``sigma_cm``, mapped affinely onto [rho_lo, rho_hi] g/cm^3, and
    given a material by density thresholds (lung below 0.6, bone above 1.4)."""
    from scipy.ndimage import gaussian_filter

    noise = rng.standard_normal((n, n, n)).astype(np.float32)
    sm = gaussian_filter(noise, sigma=sigma_cm / voxel_cm, mode="wrap")
    lo, hi = float(sm.min()), float(sm.max())
    rho = (rho_lo + (sm - lo) * (rho_hi - rho_lo) / max(hi - lo, 1e-30)).astype(np.float32)
    mat = np.full(rho.shape, MAT_WATER, dtype=np.uint8)
    mat[rho < lung_below] = MAT_LUNG
    mat[rho > bone_above] = MAT_BONE
    return Phantom((n, n, n), (voxel_cm,) * 3, mat, rho)


# ---------------------------------------------------------------------------
# Source recipes
# ---------------------------------------------------------------------------
def pencil(particle: int, energy: float, x_cm: float, y_cm: float) -> Source:
    return Source(particle, BEAM_PENCIL, energy=energy, center_cm=(x_cm, y_cm))


def square_field(particle: int, energy: float, phantom: Phantom, field_cm: float) -> Source:
    X, Y, _ = phantom.extent_cm
    return Source(particle, BEAM_SQUARE, energy=energy, center_cm=(X / 2, Y / 2),
                  field_cm=field_cm)


def point_source_phase_space(particle: int, phantom: "Phantom", n: int, seed: int,
                             source_distance_cm: float = 30.0, field_cm: float = 8.0,
                             e_lo: float = 1.0, e_hi: float = 12.0,
                             energies: Optional[np.ndarray] = None) -> Source:
    """A seeded phase space standing in for a scored one: particles on the
    z = 0 face, uniform over a square field, each aimed away from a point
    source `source_distance_cm` above the face (a diverging beam), energies
    uniform on [e_lo, e_hi] MeV, or the n given `energies`."""
    rng = np.random.default_rng(seed)
    X, Y, _ = phantom.extent_cm
    x = X / 2 + (rng.random(n) - 0.5) * field_cm
    y = Y / 2 + (rng.random(n) - 0.5) * field_cm
    d = np.stack([x - X / 2, y - Y / 2, np.full(n, source_distance_cm)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    e = e_lo + (e_hi - e_lo) * rng.random(n)
    if energies is not None:
        e = np.asarray(energies, dtype=np.float64).reshape(n)
    ps = np.column_stack([x, y, np.zeros(n), d, e])
    return Source(particle, BEAM_PHASE_SPACE, phase_space=ps)


def synthetic_6mv_spectrum(seed: int = 3, n_bins: int = 256, e_lo: float = 0.1,
                           e_hi: float = 6.0, jitter: float = 0.05
                           ) -> Tuple[np.ndarray, np.ndarray]:
    """A seeded bremsstrahlung-shaped ("6 MV-like") photon spectrum on [0.1, 6] MeV.

    Bin weights follow a thin-target Kramers-like shape (e_hi - E)/E, rolled off
    at low energy by (1 - exp(-E/0.5)) and by an analytic hardening factor
    exp(-0.15/E) that stands in for filtration, then get +-``jitter`` seeded
    multiplicative noise per bin and are normalised to sum 1.
    """
    edges = np.linspace(e_lo, e_hi, n_bins + 1)
    c = 0.5 * (edges[:-1] + edges[1:])
    w = (e_hi - c) / c * (1.0 - np.exp(-c / 0.5)) * np.exp(-0.15 / c)
    rng = np.random.default_rng(seed)
    w = w * (1.0 + jitter * (2.0 * rng.random(n_bins) - 1.0))
    w = np.maximum(w, 0.0)
    return edges.astype(np.float64), (w / w.sum()).astype(np.float64)


def draw_spectrum(edges: np.ndarray, weights: np.ndarray, n: int, seed: int) -> np.ndarray:
    """n seeded energies from a histogram spectrum: a bin by its weight, then
    uniform within the bin."""
    rng = np.random.default_rng(seed)
    k = rng.choice(len(weights), size=n, p=np.asarray(weights) / np.sum(weights))
    return edges[k] + (edges[k + 1] - edges[k]) * rng.random(n)


def polyenergetic_square(particle: int, phantom: "Phantom", field_cm: float = 10.0) -> Source:
    """A square field with a spectrum sampled on the device: photons from the
    6 MV-like spectrum, electrons flat on [1, 15] MeV (14 bins)."""
    if particle == PHOTON:
        edges, w = synthetic_6mv_spectrum()
    else:
        edges, w = np.linspace(1.0, 15.0, 15), np.full(14, 1.0 / 14)
    X, Y, _ = phantom.extent_cm
    return Source(particle, BEAM_SQUARE, center_cm=(X / 2, Y / 2), field_cm=field_cm,
                  spectrum_edges=edges, spectrum_weights=w)


def polyenergetic_phase_space(particle: int, phantom: "Phantom", n: int, seed: int) -> Source:
    """A polyenergetic phase space in random order, as a scored one would be:
    photons from the 6 MV-like spectrum, electrons uniform on [1, 15] MeV (the
    span of clinical electron energies), on a diverging 8 cm field."""
    if particle == PHOTON:
        e = draw_spectrum(*synthetic_6mv_spectrum(), n, seed + 1)
    else:
        e = 1.0 + 14.0 * np.random.default_rng(seed + 1).random(n)
    return point_source_phase_space(particle, phantom, n, seed, energies=e)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------
def config1(n_histories: int = 100_000, seed: int = 1) -> Plan:
    """2 MeV photon pencil beam along +z into 32^3 water at 0.5 cm."""
    ph = homogeneous((32, 32, 32), 0.5, MAT_WATER, 1.0)
    src = pencil(PHOTON, 2.0, 8.0, 8.0)
    return Plan("c1_water32_pencil_2MeV_photon", ph, src, n_histories, seed)


def config2(particle: int, n_histories: Optional[int] = None, n: int = 128,
            voxel_cm: float = 0.25) -> Plan:
    """15 MeV 10x10 cm^2 parallel beam on 128^3 water at 0.25 cm (32 cm cube).

    Electrons: 1e6 histories, seed 1.  Photons: 4e6 histories, seed 2.
    """
    ph = homogeneous((n, n, n), voxel_cm, MAT_WATER, 1.0)
    src = square_field(particle, 15.0, ph, 10.0)
    if particle == ELECTRON:
        return Plan("c2_water128_15MeV_electron", ph, src, n_histories or 1_000_000, 1)
    return Plan("c2_water128_15MeV_photon", ph, src, n_histories or 4_000_000, 2)


def geom2(particle: int, n_histories: Optional[int] = None, n: int = 128,
          voxel_cm: float = 0.25) -> Plan:
    """The paper's second geometry (GPUMCD §III.A): a lung box (0.26 g/cm^3) in
    water, centred on the beam axis, 4.5 cm wide; for electrons 4 cm long from
    a depth of 3 cm, for photons 6.5 cm long from 5.5 cm.  The timing-case
    beams: 15 MeV, 10x10 cm^2, 1e6 electrons (seed 1) or 4e6 photons (seed 2).
    Materials: MATERIALS."""
    X = n * voxel_cm
    z0, dz = (3.0, 4.0) if particle == ELECTRON else (5.5, 6.5)
    lo = (X / 2 - 2.25, X / 2 - 2.25, z0)
    hi = (X / 2 + 2.25, X / 2 + 2.25, z0 + dz)
    ph = box_in_water((n, n, n), voxel_cm, lo, hi, MAT_LUNG, 0.26)
    src = square_field(particle, 15.0, ph, 10.0)
    name = f"geom2_lungbox{n}_15MeV_" + ("electron" if particle == ELECTRON else "photon")
    return Plan(name, ph, src, n_histories or (1_000_000 if particle == ELECTRON else 4_000_000),
                1 if particle == ELECTRON else 2)


def geom3(particle: int, n_histories: Optional[int] = None, n: int = 128,
          voxel_cm: float = 0.25) -> Plan:
    """The paper's third geometry (GPUMCD §III.A): slabs along the beam of soft
    tissue, lung (0.26) and bone (1.85); for electrons 2 / 2 / 2 cm then
    tissue, for photons 3 / 2 / 7 cm then tissue.  Beams as in geom2.
    Materials: MATERIALS_PAPER (tissue is material 3)."""
    if particle == ELECTRON:
        slabs = [(2.0, MAT_TISSUE, 1.0), (2.0, MAT_LUNG, 0.26), (2.0, MAT_BONE, 1.85), (1e9, MAT_TISSUE, 1.0)]
    else:
        slabs = [(3.0, MAT_TISSUE, 1.0), (2.0, MAT_LUNG, 0.26), (7.0, MAT_BONE, 1.85), (1e9, MAT_TISSUE, 1.0)]
    ph = z_slabs((n, n, n), voxel_cm, slabs)
    src = square_field(particle, 15.0, ph, 10.0)
    name = f"geom3_tissue_lung_bone{n}_15MeV_" + ("electron" if particle == ELECTRON else "photon")
    return Plan(name, ph, src, n_histories or (1_000_000 if particle == ELECTRON else 4_000_000),
                1 if particle == ELECTRON else 2)


# ---------------------------------------------------------------------------
# Synthetic CT (the paper's outlook, §V, names CT-derived phantoms; no CT data
# is available, so a seeded HU volume stands in for one)
# ---------------------------------------------------------------------------
# HU -> density calibration, piecewise linear through (HU, g/cm^3) points: air,
# lung, water, then a bone branch reaching cortical bone at 1400 HU
HU_CALIBRATION = ((-1000.0, 0.0012), (-740.0, 0.26), (0.0, 1.0), (1400.0, 1.85), (3000.0, 2.8))
HU_LUNG_BELOW = -400.0  # material by HU: lung composition below, bone from HU_BONE_FROM
HU_BONE_FROM = 250.0


def hu_to_phantom(hu: np.ndarray, voxel_cm: float) -> Phantom:
    """Density by the calibration curve, material by HU thresholds: lung (water
    composition; air is lung at 0.0012 g/cm^3) below -400 HU, bone from 250 HU,
    soft tissue (MATERIALS_PAPER) between."""
    xs = np.array([p[0] for p in HU_CALIBRATION])
    ys = np.array([p[1] for p in HU_CALIBRATION])
    h = np.clip(hu.astype(np.float64), xs[0], xs[-1])
    rho = np.interp(h, xs, ys).astype(np.float32)
    mat = np.full(hu.shape, MAT_TISSUE, dtype=np.uint8)
    mat[h < HU_LUNG_BELOW] = MAT_LUNG
    mat[h >= HU_BONE_FROM] = MAT_BONE
    nz, ny, nx = hu.shape
    return Phantom((nx, ny, nz), (voxel_cm,) * 3, mat, rho)


def synthetic_ct_hu(dims: Sequence[int], voxel_cm: float, seed: int) -> np.ndarray:
    """A seeded thorax-like HU volume (z = beam depth, the body axis along y):
    an elliptic soft-tissue body (40 HU) in air, two lungs (-750 HU), a spine
    behind them and a sternum in front (1200 HU), with Gaussian noise of 20 HU
    (CT-like) everywhere inside the body."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    z = (np.arange(nz) + 0.5) * voxel_cm
    x = (np.arange(nx) + 0.5) * voxel_cm
    Z, X = np.meshgrid(z, x, indexing="ij")  # (nz, nx): the transverse slice
    cz, cx = nz * voxel_cm / 2, nx * voxel_cm / 2
    az, ax = 0.42 * nz * voxel_cm, 0.46 * nx * voxel_cm
    body = ((Z - cz) / az) ** 2 + ((X - cx) / ax) ** 2 <= 1.0
    hu2 = np.where(body, 40.0, -1000.0)
    for sx in (-1.0, 1.0):  # lungs
        lung = ((Z - cz) / (0.55 * az)) ** 2 + ((X - cx - sx * 0.45 * ax) / (0.36 * ax)) ** 2 <= 1.0
        hu2 = np.where(lung & body, -750.0, hu2)
    spine = ((Z - (cz + 0.72 * az)) / (0.14 * az)) ** 2 + ((X - cx) / (0.12 * ax)) ** 2 <= 1.0
    sternum = (np.abs(Z - (cz - 0.86 * az)) <= 0.05 * az) & (np.abs(X - cx) <= 0.12 * ax)
    hu2 = np.where((spine | sternum) & body, 1200.0, hu2)
    hu = np.repeat(hu2[:, None, :], ny, axis=1)
    noise = rng.normal(0.0, 20.0, size=hu.shape)
    return np.where(hu > -1000.0, hu + noise, hu)


def synthetic_ct(particle: int, n_histories: Optional[int] = None, dims: Sequence[int] = (128, 96, 128),
                 voxel_cm: float = 0.25, seed: int = 6) -> Plan:
    """A synthetic-CT plan: the seeded thorax HU volume through the calibration,
    a 10x10 cm^2 field entering the front (z = 0) through the sternum side: the
    6 MV-like spectrum for photons (4e6), 15 MeV for electrons (1e6)."""
    ph = hu_to_phantom(synthetic_ct_hu(dims, voxel_cm, seed), voxel_cm)
    X, Y, _ = ph.extent_cm
    if particle == PHOTON:
        edges, w = synthetic_6mv_spectrum(seed=3)
        src = Source(PHOTON, BEAM_SQUARE, center_cm=(X / 2, Y / 2), field_cm=10.0,
                     spectrum_edges=edges, spectrum_weights=w)
    else:
        src = square_field(ELECTRON, 15.0, ph, 10.0)
    name = "synthetic_ct_thorax_" + ("photon_6MV" if particle == PHOTON else "electron_15MeV")
    return Plan(name, ph, src, n_histories or (4_000_000 if particle == PHOTON else 1_000_000), seed)


def config3(n_histories: int = 10_000_000, n: int = 256, voxel_cm: float = 0.2,
            seed: int = 3) -> Plan:
    """Water / bone / lung / water slabs of 3 / 2 / 6 / rest cm on 256^3 at 0.2 cm,
    6 MV-like spectrum, 10x10 cm^2 field."""
    ph = z_slabs((n, n, n), voxel_cm,
                 [(3.0, MAT_WATER, 1.0), (2.0, MAT_BONE, 1.85), (6.0, MAT_LUNG, 0.26),
                  (1e9, MAT_WATER, 1.0)])
    edges, w = synthetic_6mv_spectrum(seed=3)
    X, Y, _ = ph.extent_cm
    src = Source(PHOTON, BEAM_SQUARE, center_cm=(X / 2, Y / 2), field_cm=10.0,
                 spectrum_edges=edges, spectrum_weights=w)
    return Plan("c3_slabs256_6MV_photon", ph, src, n_histories, seed)


@dataclasses.dataclass
class PlanSpec:
    """A batched-workload plan drawn from the config-4 distribution; the phantom
    is generated on demand because the larger ones hold tens of MB."""

    index: int
    n: int
    voxel_cm: float
    particle: int
    energy: float
    field_cm: float
    n_histories: int
    seed: int
    phantom_seed: int

    def phantom(self) -> Phantom:
        return smoothed_noise(self.n, self.voxel_cm, np.random.default_rng(self.phantom_seed))

    def plan(self, n_histories: Optional[int] = None) -> Plan:
        ph = self.phantom()
        src = square_field(self.particle, self.energy, ph, self.field_cm)
        return Plan(f"c4_plan{self.index:03d}", ph, src,
                    n_histories if n_histories is not None else self.n_histories, self.seed)


def plan_distribution(count: int, seed: int, n_lo: int = 64, n_hi: int = 256,
                      hist_lo: float = 1e5, hist_hi: float = 1e7) -> List[PlanSpec]:
    """Uneven plans: n ~ U{64..256} per axis, voxel ~ U[0.2, 0.5] cm, smoothed
    noise densities in [0.2, 2.0], photon or electron with p = 1/2, E ~ U[6, 18]
    MeV monoenergetic, square field ~ U[2, 15] cm, N ~ log-uniform [1e5, 1e7]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        vox = float(rng.uniform(0.2, 0.5))
        particle = int(rng.integers(0, 2))
        energy = float(rng.uniform(6.0, 18.0))
        field = float(rng.uniform(2.0, 15.0))
        nh = int(round(math.exp(rng.uniform(math.log(hist_lo), math.log(hist_hi)))))
        pseed = int(rng.integers(1, 2**62))
        phseed = int(rng.integers(1, 2**62))
        out.append(PlanSpec(i, n, vox, particle, energy, field, nh, pseed, phseed))
    return out


def config4(count: int = 64, seed: int = 4) -> List[PlanSpec]:
    """64 independent uneven plans for one batched persistent launch."""
    return plan_distribution(count, seed)


@dataclasses.dataclass
class Request:
    arrival_s: float
    spec: PlanSpec


def config5(count: int = 1000, seed: int = 5, rate_per_s: float = 10.0) -> List[Request]:
    """A Poisson-arrival stream of dose requests drawn from the config-4
    distribution.  ``rate_per_s`` is the mean arrival rate."""
    specs = plan_distribution(count, seed)
    rng = np.random.default_rng(seed + 1000)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    return [Request(float(t[i]), specs[i]) for i in range(count)]

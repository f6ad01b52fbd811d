"""Python access to the FP64 CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow, single-threaded
transport that checks the CUDA path.  Only tests/, ``__graft_entry__.smoke()``
and the CPU-baseline leg of bench.py may import this package.  It never
imports the CUDA library's package and the CUDA library never imports it.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["physics.c", "rng.c", "transport.c"]

MAX_EL = 16

FLAG_KERMA = 1
FLAG_FIRST_COLLISION = 2
FLAG_NO_MS = 4
FLAG_VOXEL_EMAJOR = 8  # the per-voxel electron Woodcock majorant (see oracle.h)

MEV_PER_G_TO_GY = 1.602176634e-10

_lock = threading.Lock()
_lib: Optional[C.CDLL] = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (plain C11, -O2)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    hdr = os.path.join(HERE, "oracle.h")
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(p) for p in srcs + [hdr])
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Material(C.Structure):
    _fields_ = [("n_el", C.c_int32), ("Z", C.c_int32 * MAX_EL), ("A", C.c_double * MAX_EL),
                ("w", C.c_double * MAX_EL), ("I_eV", C.c_double)]


class Physics(C.Structure):
    _fields_ = [("p_cut", C.c_double), ("e_abs", C.c_double), ("t_c", C.c_double),
                ("k_c", C.c_double), ("estepe", C.c_double), ("e_max", C.c_double),
                ("nudge_cm", C.c_double)]


class PhantomC(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("mat", C.POINTER(C.c_uint8)),
                ("rho", C.POINTER(C.c_float))]


class SourceC(C.Structure):
    _fields_ = [("particle", C.c_int32), ("beam", C.c_int32), ("energy", C.c_double),
                ("n_spec", C.c_int32), ("spec_edges", C.POINTER(C.c_double)),
                ("spec_weights", C.POINTER(C.c_double)), ("cx", C.c_double), ("cy", C.c_double),
                ("field", C.c_double), ("n_phsp", C.c_int32), ("phsp", C.POINTER(C.c_double))]


class Stats(C.Structure):
    _fields_ = [("e_incident", C.c_double), ("e_deposited", C.c_double),
                ("e_escaped", C.c_double), ("e_rest", C.c_double), ("e_cut_photon", C.c_double),
                ("e_cut_electron", C.c_double), ("track_length_cm", C.c_double),
                ("n_histories", C.c_uint64), ("n_photon_real", C.c_uint64),
                ("n_photon_fict", C.c_uint64), ("n_compton", C.c_uint64), ("n_photo", C.c_uint64),
                ("n_pair", C.c_uint64), ("n_e_steps", C.c_uint64), ("n_hard_real", C.c_uint64),
                ("n_hard_fict", C.c_uint64), ("n_moller", C.c_uint64), ("n_brem", C.c_uint64),
                ("n_electrons", C.c_uint64), ("n_photons", C.c_uint64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_DP = C.POINTER(C.c_double)
_MP = C.POINTER(Material)


def lib() -> C.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            d = C.c_double
            for name in ("om_sigma_kn",):
                getattr(L, name).argtypes = [d]
                getattr(L, name).restype = d
            L.om_kn_dsigma_domega.argtypes = [d, d]
            L.om_kn_dsigma_domega.restype = d
            L.om_electron_density.argtypes = [_MP]
            L.om_electron_density.restype = d
            for name in ("om_mu_compton", "om_mu_photo", "om_mu_pair", "om_mu_total", "om_s_col",
                         "om_s_rad", "om_ms_lambda1_inv"):
                getattr(L, name).argtypes = [_MP, d]
                getattr(L, name).restype = d
            for name in ("om_l_col", "om_l_rad", "om_sigma_moller", "om_sigma_brem",
                         "om_brem_dsigma_dk"):
                getattr(L, name).argtypes = [_MP, d, d]
                getattr(L, name).restype = d
            L.om_moller_dsigma_deps.argtypes = [d, d]
            L.om_moller_dsigma_deps.restype = d
            L.om_ms_screening.argtypes = [C.c_int, d]
            L.om_ms_screening.restype = d
            L.om_ms_mean_mu.argtypes = [d]
            L.om_ms_mean_mu.restype = d
            L.om_ms_solve_a.argtypes = [d]
            L.om_ms_solve_a.restype = d
            L.om_sample_kn.argtypes = [d, C.c_int64, C.c_uint64, _DP, _DP]
            L.om_sample_sauter.argtypes = [d, C.c_int64, C.c_uint64, _DP]
            L.om_sample_moller.argtypes = [d, d, C.c_int64, C.c_uint64, _DP]
            L.om_sample_brem.argtypes = [_MP, d, d, C.c_int64, C.c_uint64, _DP]
            L.om_sample_ms.argtypes = [d, C.c_int64, C.c_uint64, _DP]
            L.om_sample_spectrum.argtypes = [C.c_int32, _DP, _DP, C.c_int64, C.c_uint64, _DP]
            L.om_primary_energies.argtypes = [C.POINTER(SourceC), C.c_uint64, C.c_uint64,
                                              C.c_uint64, _DP]
            L.om_primary_energies.restype = C.c_int32
            L.om_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
            L.om_rotate.argtypes = [_DP, d, d, _DP]
            L.om_compton_kinematics.argtypes = [d, _DP, d, d, d, _DP, _DP, _DP]
            L.om_moller_kinematics.argtypes = [d, d, _DP]
            L.om_simulate.argtypes = [_MP, C.c_int32, C.POINTER(Physics), C.POINTER(PhantomC),
                                      C.POINTER(SourceC), C.c_uint64, C.c_uint64, C.c_uint64,
                                      C.c_uint32, _DP, _DP, C.POINTER(Stats)]
            L.om_simulate.restype = C.c_int32
            L.om_first_interaction_z.argtypes = [_MP, C.c_int32, C.POINTER(Physics),
                                                 C.POINTER(PhantomC), C.POINTER(SourceC),
                                                 C.c_int64, C.c_uint64, _DP,
                                                 C.POINTER(C.c_uint64)]
            L.om_first_interaction_z.restype = C.c_int32
            _lib = L
        return _lib


# ---------------------------------------------------------------------------
# Conversions from the workload objects (workloads/).
# ---------------------------------------------------------------------------
def material(m) -> Material:
    out = Material()
    Z, A, w = m.Z, m.A, m.w
    out.n_el = len(Z)
    for i in range(len(Z)):
        out.Z[i] = Z[i]
        out.A[i] = A[i]
        out.w[i] = w[i]
    out.I_eV = m.I_eV
    return out


def materials(mats) -> C.Array:
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i] = material(m)
    return arr


def physics(p) -> Physics:
    return Physics(p.p_cut, p.e_abs, p.t_c, p.k_c, p.estepe, p.e_max, p.nudge_cm)


class _Keep:
    """Holds numpy buffers alive while a C struct points into them."""

    def __init__(self):
        self.refs = []


def phantom(ph, keep: _Keep) -> PhantomC:
    mat = np.ascontiguousarray(ph.mat, dtype=np.uint8).ravel()
    rho = np.ascontiguousarray(ph.rho, dtype=np.float32).ravel()
    keep.refs += [mat, rho]
    nx, ny, nz = ph.dims
    dx, dy, dz = ph.voxel_cm
    return PhantomC(nx, ny, nz, dx, dy, dz, mat.ctypes.data_as(C.POINTER(C.c_uint8)),
                    rho.ctypes.data_as(C.POINTER(C.c_float)))


def source(src, keep: _Keep) -> SourceC:
    """The C source.  Energy grouping (§IV) changes no sample: a grouped
    spectrum or phase space starts every history as an ungrouped one does (the
    grouping orders which histories run together, and the oracle runs them one
    after another), so the flag is not passed on."""
    s = SourceC()
    s.particle = src.particle
    s.beam = src.beam
    s.energy = src.energy
    s.cx, s.cy = src.center_cm
    s.field = src.field_cm
    if src.spectrum_edges is not None:
        e = np.ascontiguousarray(src.spectrum_edges, dtype=np.float64)
        w = np.ascontiguousarray(src.spectrum_weights, dtype=np.float64)
        keep.refs += [e, w]
        s.n_spec = len(w)
        s.spec_edges = e.ctypes.data_as(_DP)
        s.spec_weights = w.ctypes.data_as(_DP)
    else:
        s.n_spec = 0
    ps = getattr(src, "phase_space", None)
    if ps is not None:
        a = np.ascontiguousarray(ps, dtype=np.float64).reshape(-1, 7)
        keep.refs.append(a)
        s.n_phsp = len(a)
        s.phsp = a.ctypes.data_as(_DP)
    else:
        s.n_phsp = 0
    return s


# ---------------------------------------------------------------------------
# Transport runs.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class OracleResult:
    n_histories: int
    sum_e: np.ndarray  # MeV, per voxel, summed over histories
    sum_e2: np.ndarray  # MeV^2
    stats: dict
    seconds: float = 0.0
    cores: int = 1

    def dose_gy(self, ph) -> np.ndarray:
        """Mean dose per history in Gy (MeV/g x 1.602176634e-10)."""
        mass = ph.rho.ravel().astype(np.float64) * float(np.prod(ph.voxel_cm))
        with np.errstate(divide="ignore", invalid="ignore"):
            d = np.where(mass > 0, self.sum_e / self.n_histories / mass, 0.0)
        return d * MEV_PER_G_TO_GY

    def sigma_gy(self, ph) -> np.ndarray:
        """History-by-history standard error of the mean dose (GPUMCD §II.D)."""
        n = self.n_histories
        mean = self.sum_e / n
        var = np.maximum(self.sum_e2 / n - mean * mean, 0.0) / max(n - 1, 1)
        mass = ph.rho.ravel().astype(np.float64) * float(np.prod(ph.voxel_cm))
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(mass > 0, np.sqrt(var) / mass, 0.0)
        return s * MEV_PER_G_TO_GY


def simulate_range(mats, phys, ph, src, h0: int, h1: int, seed: int, flags: int = 0):
    """One single-threaded oracle call over histories [h0, h1)."""
    L = lib()
    keep = _Keep()
    marr = materials(mats)
    pc = phantom(ph, keep)
    sc = source(src, keep)
    pp = physics(phys)
    s1 = np.zeros(ph.nvox, dtype=np.float64)
    s2 = np.zeros(ph.nvox, dtype=np.float64)
    st = Stats()
    rc = L.om_simulate(marr, len(mats), C.byref(pp), C.byref(pc), C.byref(sc), h0, h1, seed,
                       flags, s1.ctypes.data_as(_DP), s2.ctypes.data_as(_DP), C.byref(st))
    if rc != 0:
        raise RuntimeError(f"om_simulate failed with status {rc}")
    return s1, s2, st.as_dict()


def _worker(args):
    mats, phys, ph, src, h0, h1, seed, flags = args
    return simulate_range(mats, phys, ph, src, h0, h1, seed, flags)


def simulate(mats, phys, ph, src, n_histories: int, seed: int, flags: int = 0,
             processes: int = 1, hist_begin: int = 0) -> OracleResult:
    """Runs histories [hist_begin, hist_begin + n) of the oracle.  With
    processes > 1 the history range is split over spawned worker processes;
    histories are independent and their random streams are keyed by the history
    index, so the split does not change the result beyond FP64 summation order."""
    import time

    t0 = time.perf_counter()
    if processes <= 1 or n_histories < 2 * processes:
        s1, s2, st = simulate_range(mats, phys, ph, src, hist_begin, hist_begin + n_histories,
                                    seed, flags)
        procs = 1
    else:
        import multiprocessing as mp

        cuts = np.linspace(hist_begin, hist_begin + n_histories, processes + 1).astype(np.int64)
        jobs = [(mats, phys, ph, src, int(cuts[i]), int(cuts[i + 1]), seed, flags)
                for i in range(processes)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes) as pool:
            parts = pool.map(_worker, jobs)
        s1 = sum(p[0] for p in parts)
        s2 = sum(p[1] for p in parts)
        st = {k: sum(p[2][k] for p in parts) for k in parts[0][2]}
        procs = processes
    return OracleResult(n_histories, s1, s2, st, time.perf_counter() - t0, procs)


def simulate_parts(mats, phys, ph, src, n_histories: int, seed: int, parts: int,
                   processes: int = 1, flags: int = 0):
    """Histories [0, n) split into `parts` equal, independent ranges (for
    sample-variance estimates of any aggregate), run over one pool of spawned
    workers.  Returns one OracleResult per part."""
    import multiprocessing as mp
    import time

    t0 = time.perf_counter()
    cuts = np.linspace(0, n_histories, parts + 1).astype(np.int64)
    per_part = max(1, processes // parts)
    jobs, owner = [], []
    for i in range(parts):
        sub = np.linspace(cuts[i], cuts[i + 1], per_part + 1).astype(np.int64)
        for j in range(per_part):
            if sub[j + 1] > sub[j]:
                jobs.append((mats, phys, ph, src, int(sub[j]), int(sub[j + 1]), seed, flags))
                owner.append(i)
    with mp.get_context("spawn").Pool(max(1, min(processes, len(jobs)))) as pool:
        outs = pool.map(_worker, jobs)
    res = []
    for i in range(parts):
        mine = [o for o, k in zip(outs, owner) if k == i]
        s1 = sum(o[0] for o in mine)
        s2 = sum(o[1] for o in mine)
        st = {k: sum(o[2][k] for o in mine) for k in mine[0][2]}
        res.append(OracleResult(int(cuts[i + 1] - cuts[i]), s1, s2, st,
                                time.perf_counter() - t0, processes))
    return res


def primary_energies(src, h0: int, h1: int, seed: int) -> np.ndarray:
    """The primary energies (MeV) of histories [h0, h1), drawn as the
    transport draws them."""
    L = lib()
    keep = _Keep()
    sc = source(src, keep)
    out = np.zeros(h1 - h0, dtype=np.float64)
    if L.om_primary_energies(C.byref(sc), h0, h1, seed, out.ctypes.data_as(_DP)) != 0:
        raise RuntimeError("om_primary_energies failed")
    return out


def first_interaction_z(mats, phys, ph, src, n: int, seed: int):
    L = lib()
    keep = _Keep()
    marr = materials(mats)
    pc = phantom(ph, keep)
    sc = source(src, keep)
    pp = physics(phys)
    z = np.zeros(n, dtype=np.float64)
    nf = C.c_uint64(0)
    rc = L.om_first_interaction_z(marr, len(mats), C.byref(pp), C.byref(pc), C.byref(sc), n,
                                  seed, z.ctypes.data_as(_DP), C.byref(nf))
    if rc != 0:
        raise RuntimeError(f"om_first_interaction_z failed with status {rc}")
    return z, int(nf.value)


# ---------------------------------------------------------------------------
# Point evaluations and samplers.
# ---------------------------------------------------------------------------
def xs(name: str, mat, *args) -> float:
    L = lib()
    m = material(mat)
    return getattr(L, "om_" + name)(C.byref(m), *args)


def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.om_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def sample(kind: str, n: int, seed: int, *params):
    L = lib()
    out = np.zeros(n, dtype=np.float64)
    p = out.ctypes.data_as(_DP)
    if kind == "kn":
        eps = np.zeros(n, dtype=np.float64)
        L.om_sample_kn(params[0], n, seed, p, eps.ctypes.data_as(_DP))
        return out, eps
    if kind == "sauter":
        L.om_sample_sauter(params[0], n, seed, p)
    elif kind == "moller":
        L.om_sample_moller(params[0], params[1], n, seed, p)
    elif kind == "brem":
        m = material(params[0])
        L.om_sample_brem(C.byref(m), params[1], params[2], n, seed, p)
    elif kind == "ms":
        L.om_sample_ms(params[0], n, seed, p)
    elif kind == "spectrum":
        edges = np.ascontiguousarray(params[0], dtype=np.float64)
        w = np.ascontiguousarray(params[1], dtype=np.float64)
        L.om_sample_spectrum(len(w), edges.ctypes.data_as(_DP), w.ctypes.data_as(_DP), n, seed, p)
    else:
        raise ValueError(kind)
    return out


def rotate(u, cos_t: float, phi: float) -> np.ndarray:
    """The transport's rotation of unit vector u by polar angle acos(cos_t)
    and azimuth phi."""
    L = lib()
    a = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    L.om_rotate(a.ctypes.data_as(_DP), cos_t, phi, out.ctypes.data_as(_DP))
    return out


def compton_kinematics(E: float, u, cos_t: float, eps: float, phi: float):
    """The transport's Compton kinematics: (photon direction, recoil electron
    direction, E', T)."""
    L = lib()
    a = np.ascontiguousarray(u, dtype=np.float64)
    u1, ue, o = np.zeros(3), np.zeros(3), np.zeros(2)
    L.om_compton_kinematics(E, a.ctypes.data_as(_DP), cos_t, eps, phi, u1.ctypes.data_as(_DP),
                            ue.ctypes.data_as(_DP), o.ctypes.data_as(_DP))
    return u1, ue, float(o[0]), float(o[1])


def moller_kinematics(T: float, eps: float):
    """The transport's Moller kinematics: (T_knock-on, T_scattered,
    cos_knock-on, cos_scattered)."""
    L = lib()
    o = np.zeros(4)
    L.om_moller_kinematics(T, eps, o.ctypes.data_as(_DP))
    return tuple(float(x) for x in o)

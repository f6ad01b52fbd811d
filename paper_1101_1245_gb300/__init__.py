"""Python binding of the gpumcd C ABI (include/gpumcd.h).

Argument marshalling only: every step of the transport runs in the CUDA
library (paper_1101_1245_gb300/libgpumcd.so).  There is no CPU fallback; if the
library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

MAX_MATERIALS = 4
MAX_ELEMENTS = 16
MAX_PLANS_PER_RUN = 64
MAX_INFLIGHT = 2
ENERGY_QUANTUM_MEV = 1.0 / 67108864.0
PHOTON, ELECTRON = 0, 1
BEAM_PENCIL, BEAM_SQUARE, BEAM_PHASE_SPACE = 0, 1, 2
ENERGY_UNGROUPED, ENERGY_GROUPED = 0, 1  # gpumcd_source.energy_grouping
LAUNCH_WARP_AGGREGATE = 1
LAUNCH_PROFILE = 2
LAUNCH_GRAPH = 4
LAUNCH_KERMA = 8
# refill_period of the launch: refill empty lanes only when the whole warp is empty
REFILL_WHEN_EMPTY = 0xFFFFFFFF
PARTICLE_TYPES = ("photon", "electron")

STATUS = {
    0: "ok", -1: "invalid argument", -2: "device out of memory", -3: "CUDA error",
    -4: "particle queue overflow", -5: "device wait timed out", -6: "unknown id",
    -7: "HBM budget exceeded", -8: "call out of order",
}
OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_QUEUE_OVERFLOW, ERR_TIMEOUT, ERR_NOT_FOUND, \
    ERR_BUDGET, ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7, -8


class GpumcdError(RuntimeError):
    def __init__(self, status: int, call: str):
        super().__init__(f"{call}: {STATUS.get(status, 'unknown')} ({status})")
        self.status = status


class Material(C.Structure):
    _fields_ = [("n_elements", C.c_int32), ("Z", C.c_int32 * MAX_ELEMENTS),
                ("A", C.c_double * MAX_ELEMENTS), ("w", C.c_double * MAX_ELEMENTS),
                ("I_eV", C.c_double)]


class Physics(C.Structure):
    _fields_ = [("p_cut", C.c_double), ("e_abs", C.c_double), ("t_c", C.c_double),
                ("k_c", C.c_double), ("estepe", C.c_double), ("e_max", C.c_double),
                ("nudge_cm", C.c_double)]


class Source(C.Structure):
    _fields_ = [("particle", C.c_int32), ("beam", C.c_int32), ("energy_mev", C.c_double),
                ("n_spectrum", C.c_int32), ("spectrum_edges", C.POINTER(C.c_double)),
                ("spectrum_weights", C.POINTER(C.c_double)), ("center_cm", C.c_double * 2),
                ("field_cm", C.c_double), ("n_phase_space", C.c_int32),
                ("phase_space", C.POINTER(C.c_double)), ("energy_grouping", C.c_int32)]


class Launch(C.Structure):
    _fields_ = [("block_threads", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("stack_capacity", C.c_uint32), ("switch_high", C.c_uint32),
                ("refill_low", C.c_uint32), ("chunk", C.c_uint32),
                ("overflow_capacity", C.c_uint32), ("flags", C.c_uint32),
                ("refill_period", C.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class RunStats(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("e_incident", C.c_uint64),
                ("e_deposited", C.c_uint64), ("e_escaped", C.c_uint64), ("e_rest", C.c_uint64),
                ("n_photon_events", C.c_uint64), ("n_photon_real", C.c_uint64),
                ("n_compton", C.c_uint64), ("n_photo", C.c_uint64), ("n_pair", C.c_uint64),
                ("n_electron_steps", C.c_uint64), ("n_hard_real", C.c_uint64),
                ("n_hard_fict", C.c_uint64), ("n_moller", C.c_uint64), ("n_brem", C.c_uint64),
                ("n_photons", C.c_uint64), ("n_electrons", C.c_uint64), ("n_overflow", C.c_uint64),
                ("n_spilled", C.c_uint64),
                ("n_sampler_capped", C.c_uint64),
                ("n_launches", C.c_uint32), ("n_batches", C.c_uint32),
                ("transport_ms", C.c_double), ("d_max_gy", C.c_double), ("s_thr", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_I32 = C.c_int32
_U64 = C.c_uint64
_D = C.c_double
_ST = C.c_int32
_CTX = C.c_void_p

# name -> (restype, argtypes); the names and order follow include/gpumcd.h
SIGNATURES = {
    "gpumcd_status_string": (C.c_char_p, [_ST]),
    "gpumcd_init": (_ST, [C.POINTER(_CTX), _I32, _U64]),
    "gpumcd_destroy": (_ST, [_CTX]),
    "gpumcd_load_materials": (_ST, [_CTX, C.POINTER(Material), _I32, C.POINTER(Physics)]),
    "gpumcd_create_phantom": (_ST, [_CTX, C.POINTER(_I32), C.POINTER(_D), _P, _P, C.POINTER(_I32)]),
    "gpumcd_create_phantom_device": (_ST, [_CTX, C.POINTER(_I32), C.POINTER(_D), _P, _P, _P,
                                           C.POINTER(_I32)]),
    "gpumcd_destroy_phantom": (_ST, [_CTX, _I32]),
    "gpumcd_simulate": (_ST, [_CTX, _I32, C.POINTER(Source), _U64, _U64, _D, _P, _P,
                              C.POINTER(RunStats)]),
    "gpumcd_simulate_device": (_ST, [_CTX, _I32, C.POINTER(Source), _U64, _U64, _D, _P, _P, _P,
                                     C.POINTER(RunStats)]),
    "gpumcd_plan_open": (_ST, [_CTX, _I32, C.POINTER(Source), _U64, C.c_uint32, C.POINTER(_I32)]),
    "gpumcd_plan_close": (_ST, [_CTX, _I32]),
    "gpumcd_plan_reset": (_ST, [_CTX, _I32, _U64, _P]),
    "gpumcd_run": (_ST, [_CTX, _I32, C.POINTER(_I32), C.POINTER(_U64), _P]),
    "gpumcd_submit": (_ST, [_CTX, _I32, C.POINTER(_I32), C.POINTER(_U64), C.POINTER(_I32)]),
    "gpumcd_poll": (_ST, [_CTX, _I32, C.POINTER(_I32)]),
    "gpumcd_wait": (_ST, [_CTX, _I32]),
    "gpumcd_plan_result": (_ST, [_CTX, _I32, _D, _P, _P, _P, C.POINTER(RunStats)]),
    "gpumcd_plan_result_host": (_ST, [_CTX, _I32, _D, _P, _P, C.POINTER(RunStats)]),
    "gpumcd_run_to_uncertainty": (_ST, [_CTX, _I32, C.POINTER(_I32), C.POINTER(_U64), C.POINTER(_U64), _D, _D,
                                        _P, C.POINTER(_U64), C.POINTER(_D), C.POINTER(C.c_uint32),
                                        C.POINTER(_D), C.POINTER(C.c_uint32)]),
    "gpumcd_plan_histories": (_ST, [_CTX, _I32, C.POINTER(_U64)]),
    "gpumcd_plan_result_noalloc": (_ST, [_CTX, _I32, _D, _P, _P, _P, C.POINTER(RunStats)]),
    "gpumcd_memory": (_ST, [_CTX, C.POINTER(_U64), C.POINTER(_U64)]),
    "gpumcd_set_launch": (_ST, [_CTX, C.POINTER(Launch)]),
    "gpumcd_get_launch": (_ST, [_CTX, C.POINTER(Launch)]),
    "gpumcd_get_tables": (_ST, [_CTX, _I32, _P, C.POINTER(_I32)]),
    "gpumcd_debug_sample": (_ST, [_CTX, _I32, _D, _I32, C.POINTER(Source), _U64, _U64, _P]),
    "gpumcd_debug_counters": (_ST, [_CTX, _P, C.POINTER(_I32)]),
    "gpumcd_debug_philox": (_ST, [_CTX, _P, _P, _U64, _I32, _P]),
    "gpumcd_debug_majorants": (_ST, [_CTX, _I32, _P, _P]),
}

_lock = threading.Lock()
_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """Loads (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(status: int, call: str) -> None:
    if status != OK:
        raise GpumcdError(status, call)


def status_string(status: int) -> str:
    return lib().gpumcd_status_string(status).decode()


# ---------------------------------------------------------------------------
# Conversions from the workload objects
# ---------------------------------------------------------------------------
def material(m) -> Material:
    out = Material()
    out.n_elements = len(m.Z)
    for i, (z, a, w) in enumerate(zip(m.Z, m.A, m.w)):
        out.Z[i], out.A[i], out.w[i] = z, a, w
    out.I_eV = m.I_eV
    return out


def physics(p) -> Physics:
    return Physics(p.p_cut, p.e_abs, p.t_c, p.k_c, p.estepe, p.e_max, p.nudge_cm)


class _SourceBox:
    """A ctypes Source plus the arrays it points into."""

    def __init__(self, src):
        self.s = Source()
        self.s.particle = src.particle
        self.s.beam = src.beam
        self.s.energy_mev = src.energy
        self.s.center_cm[0], self.s.center_cm[1] = src.center_cm
        self.s.field_cm = src.field_cm
        self.keep = []
        if src.spectrum_edges is not None:
            e = np.ascontiguousarray(src.spectrum_edges, dtype=np.float64)
            w = np.ascontiguousarray(src.spectrum_weights, dtype=np.float64)
            self.keep = [e, w]
            self.s.n_spectrum = len(w)
            self.s.spectrum_edges = e.ctypes.data_as(C.POINTER(C.c_double))
            self.s.spectrum_weights = w.ctypes.data_as(C.POINTER(C.c_double))
        ps = getattr(src, "phase_space", None)
        if ps is not None:
            a = np.ascontiguousarray(ps, dtype=np.float64).reshape(-1, 7)
            self.keep.append(a)
            self.s.n_phase_space = len(a)
            self.s.phase_space = a.ctypes.data_as(C.POINTER(C.c_double))
        self.s.energy_grouping = getattr(src, "energy_grouping", ENERGY_UNGROUPED)


@dataclasses.dataclass
class Result:
    dose: np.ndarray
    sigma: np.ndarray
    stats: dict


class Context:
    """A gpumcd context on one CUDA device (gpumcd_init ... gpumcd_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._L = lib()
        h = _CTX()
        _check(self._L.gpumcd_init(C.byref(h), device, hbm_budget_bytes), "gpumcd_init")
        self.h = h
        self.device = device

    def close(self) -> None:
        if getattr(self, "h", None):
            self._L.gpumcd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    # ---- setup -------------------------------------------------------------
    def load_materials(self, mats: Sequence, phys) -> None:
        arr = (Material * len(mats))(*[material(m) for m in mats])
        pp = physics(phys)
        _check(self._L.gpumcd_load_materials(self.h, arr, len(mats), C.byref(pp)),
               "gpumcd_load_materials")

    def create_phantom(self, ph) -> int:
        dims = (_I32 * 3)(*ph.dims)
        vox = (_D * 3)(*ph.voxel_cm)
        mat = np.ascontiguousarray(ph.mat, dtype=np.uint8)
        rho = np.ascontiguousarray(ph.rho, dtype=np.float32)
        pid = _I32()
        _check(self._L.gpumcd_create_phantom(self.h, dims, vox, mat.ctypes.data, rho.ctypes.data,
                                             C.byref(pid)), "gpumcd_create_phantom")
        return pid.value

    def create_phantom_device(self, dims, voxel_cm, mat_ptr: int, rho_ptr: int,
                              stream: int = 0) -> int:
        d = (_I32 * 3)(*dims)
        v = (_D * 3)(*voxel_cm)
        pid = _I32()
        _check(self._L.gpumcd_create_phantom_device(self.h, d, v, mat_ptr, rho_ptr, stream or None,
                                                    C.byref(pid)),
               "gpumcd_create_phantom_device")
        return pid.value

    def destroy_phantom(self, pid: int) -> None:
        _check(self._L.gpumcd_destroy_phantom(self.h, pid), "gpumcd_destroy_phantom")

    # ---- one-shot runs -----------------------------------------------------
    def simulate(self, pid: int, src, n_histories: int, seed: int, target_rel_unc: float = 0.0,
                 nvox: Optional[int] = None, want_dose: bool = True, out=None) -> Result:
        """gpumcd_simulate with host outputs: new arrays, or ``out`` = (dose, sigma),
        two C-contiguous float64 arrays of nvox entries the caller owns (for
        example views of pinned host memory)."""
        box = _SourceBox(src)
        st = RunStats()
        if out is not None:
            dose, sig = out
            for a in (dose, sig):
                if a.dtype != np.float64 or not a.flags.c_contiguous or (nvox and a.size != nvox):
                    raise ValueError("out arrays must be C-contiguous float64 of nvox entries")
            want_dose = True
        else:
            dose = np.zeros(nvox, dtype=np.float64) if want_dose else None
            sig = np.zeros(nvox, dtype=np.float64) if want_dose else None
        _check(self._L.gpumcd_simulate(self.h, pid, C.byref(box.s), n_histories, seed, target_rel_unc,
                                       dose.ctypes.data if want_dose else None,
                                       sig.ctypes.data if want_dose else None, C.byref(st)),
               "gpumcd_simulate")
        return Result(dose, sig, st.as_dict())

    def simulate_device(self, pid: int, src, n_histories: int, seed: int, dose_ptr: int,
                        sigma_ptr: int, stream: int = 0, target_rel_unc: float = 0.0) -> dict:
        box = _SourceBox(src)
        st = RunStats()
        _check(self._L.gpumcd_simulate_device(self.h, pid, C.byref(box.s), n_histories, seed,
                                              target_rel_unc, dose_ptr or None, sigma_ptr or None,
                                              stream or None, C.byref(st)),
               "gpumcd_simulate_device")
        return st.as_dict()

    # ---- plans ---------------------------------------------------------------
    def plan_open(self, pid: int, src, seed: int, n_batches: int = 32) -> int:
        box = _SourceBox(src)
        out = _I32()
        _check(self._L.gpumcd_plan_open(self.h, pid, C.byref(box.s), seed, n_batches, C.byref(out)),
               "gpumcd_plan_open")
        return out.value

    def plan_close(self, plan: int) -> None:
        _check(self._L.gpumcd_plan_close(self.h, plan), "gpumcd_plan_close")

    def plan_reset(self, plan: int, seed: int, stream: int = 0) -> None:
        _check(self._L.gpumcd_plan_reset(self.h, plan, seed, stream or None), "gpumcd_plan_reset")

    def run(self, plans: Sequence[int], n_histories: Sequence[int], stream: int = 0) -> None:
        ids = (_I32 * len(plans))(*plans)
        ns = (_U64 * len(plans))(*n_histories)
        _check(self._L.gpumcd_run(self.h, len(plans), ids, ns, stream or None), "gpumcd_run")

    def submit(self, plans: Sequence[int], n_histories: Sequence[int]) -> int:
        """Asynchronous run: enqueues the launch sequence and returns its ticket."""
        ids = (_I32 * len(plans))(*plans)
        ns = (_U64 * len(plans))(*n_histories)
        t = _I32()
        _check(self._L.gpumcd_submit(self.h, len(plans), ids, ns, C.byref(t)), "gpumcd_submit")
        return t.value

    def poll(self, ticket: int) -> bool:
        """True once the ticket's sequence has finished (raising on its failure)."""
        d = _I32()
        _check(self._L.gpumcd_poll(self.h, ticket, C.byref(d)), "gpumcd_poll")
        return bool(d.value)

    def wait(self, ticket: int) -> None:
        _check(self._L.gpumcd_wait(self.h, ticket), "gpumcd_wait")

    def plan_result(self, plan: int, threshold: float = 0.5, dose_ptr: int = 0,
                    sigma_ptr: int = 0, stream: int = 0) -> dict:
        st = RunStats()
        _check(self._L.gpumcd_plan_result(self.h, plan, threshold, dose_ptr or None,
                                          sigma_ptr or None, stream or None, C.byref(st)),
               "gpumcd_plan_result")
        return st.as_dict()

    def plan_result_host(self, plan: int, threshold: float = 0.5, dose: Optional[np.ndarray] = None,
                         sigma: Optional[np.ndarray] = None) -> dict:
        """gpumcd_plan_result_host into caller-owned C-contiguous float64 host
        arrays of nvox entries (for example views of pinned memory)."""
        for a in (dose, sigma):
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
                raise ValueError("host outputs must be C-contiguous float64 arrays")
        st = RunStats()
        _check(self._L.gpumcd_plan_result_host(self.h, plan, threshold,
                                               dose.ctypes.data if dose is not None else None,
                                               sigma.ctypes.data if sigma is not None else None,
                                               C.byref(st)), "gpumcd_plan_result_host")
        return st.as_dict()

    def run_to_uncertainty(self, plans: Sequence[int], first_histories: Sequence[int],
                           max_histories: Sequence[int], target: float, threshold: float = 0.5,
                           stream: int = 0) -> dict:
        """gpumcd_run_to_uncertainty: the plans' total histories, final s, the
        rounds run, the device time of their transport launches and the launch
        sequences they took."""
        k = len(plans)
        ids = (_I32 * k)(*plans)
        first = (_U64 * k)(*first_histories)
        mx = (_U64 * k)(*max_histories)
        h = (_U64 * k)()
        s = (_D * k)()
        r = C.c_uint32()
        ms = _D()
        q = C.c_uint32()
        _check(self._L.gpumcd_run_to_uncertainty(self.h, k, ids, first, mx, target, threshold, stream or None,
                                                 h, s, C.byref(r), C.byref(ms), C.byref(q)),
               "gpumcd_run_to_uncertainty")
        return {"histories": list(h), "s_thr": list(s), "rounds": r.value, "transport_ms": ms.value,
                "sequences": q.value}

    def plan_histories(self, plan: int) -> int:
        h = _U64()
        _check(self._L.gpumcd_plan_histories(self.h, plan, C.byref(h)), "gpumcd_plan_histories")
        return h.value

    def memory(self) -> Tuple[int, int]:
        u, b = _U64(), _U64()
        _check(self._L.gpumcd_memory(self.h, C.byref(u), C.byref(b)), "gpumcd_memory")
        return u.value, b.value

    # ---- tuning and diagnostics ------------------------------------------
    def set_launch(self, **kw) -> None:
        cur = self.get_launch()
        cur.update(kw)
        L = Launch(**cur)
        _check(self._L.gpumcd_set_launch(self.h, C.byref(L)), "gpumcd_set_launch")

    def get_launch(self) -> dict:
        L = Launch()
        _check(self._L.gpumcd_get_launch(self.h, C.byref(L)), "gpumcd_get_launch")
        return L.as_dict()

    def get_tables(self, which: int) -> np.ndarray:
        n = _I32()
        _check(self._L.gpumcd_get_tables(self.h, which, None, C.byref(n)), "gpumcd_get_tables")
        out = np.zeros(n.value, dtype=np.float32)
        _check(self._L.gpumcd_get_tables(self.h, which, out.ctypes.data, C.byref(n)),
               "gpumcd_get_tables")
        return out

    def debug_sample(self, kind: int, p0: float, n: int, seed: int, material: int = 0,
                     src=None) -> np.ndarray:
        out = np.zeros(n, dtype=np.float32)
        box = _SourceBox(src) if src is not None else None
        _check(self._L.gpumcd_debug_sample(self.h, kind, p0, material,
                                           C.byref(box.s) if box else None, n, seed,
                                           out.ctypes.data), "gpumcd_debug_sample")
        return out

    def debug_counters(self) -> np.ndarray:
        n = _I32()
        _check(self._L.gpumcd_debug_counters(self.h, None, C.byref(n)), "gpumcd_debug_counters")
        out = np.zeros(n.value, dtype=np.uint64)
        _check(self._L.gpumcd_debug_counters(self.h, out.ctypes.data, C.byref(n)),
               "gpumcd_debug_counters")
        return out

    def profile(self) -> dict:
        """Per-particle-type cycle profile of the last run (needs LAUNCH_PROFILE):
        warp-cycles of the event passes, passes, lane occupancy, refill cycles."""
        c = self.debug_counters().astype(np.float64)
        base = 15
        cyc, it, lanes = c[base:base + 2], c[base + 2:base + 4], c[base + 4:base + 6]
        out = {}
        for i, name in enumerate(PARTICLE_TYPES):
            out[name] = {"cycles": cyc[i], "iterations": it[i],
                         "lane_occupancy": lanes[i] / (32 * it[i]) if it[i] else 0.0,
                         "cycles_per_iteration": cyc[i] / it[i] if it[i] else 0.0}
        out["refill_cycles"], out["switches"] = c[base + 6], c[base + 7]
        return out

    def debug_majorants(self, phantom_id: int) -> Tuple[np.ndarray, np.ndarray]:
        """The phantom's majorant tables (photon | electron, 1/cm, float32) and
        per-material maximum densities (g/cm^3)."""
        maj = np.zeros(1024, dtype=np.float32)
        rho = np.zeros(MAX_MATERIALS, dtype=np.float32)
        _check(self._L.gpumcd_debug_majorants(self.h, int(phantom_id), maj.ctypes.data, rho.ctypes.data),
               "gpumcd_debug_majorants")
        return maj, rho

    def debug_philox(self, ctr: np.ndarray, key: Sequence[int], use_curand: bool = False
                     ) -> np.ndarray:
        ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
        k = np.asarray(key, dtype=np.uint32)
        out = np.zeros_like(ctr)
        _check(self._L.gpumcd_debug_philox(self.h, ctr.ctypes.data, k.ctypes.data, len(ctr),
                                           int(use_curand), out.ctypes.data), "gpumcd_debug_philox")
        return out


def engine(device: int = 0, mats=None, phys=None, hbm_budget_bytes: int = 0) -> Context:
    """A context with the standard materials and transport parameters loaded."""
    import workloads as W

    ctx = Context(device, hbm_budget_bytes)
    ctx.load_materials(mats if mats is not None else W.MATERIALS,
                       phys if phys is not None else W.DEFAULT_PHYSICS)
    return ctx

"""Roofline of the transport kernel: SM instruction issue.

Transport is neither a dense contraction nor HBM-bound; it is bound by the
instruction issue of the SMs (FP32/INT ALU work, divergence and latency).  The
ceiling is 4 warp-instructions per clock per SM (one per SM sub-partition),
times the SM count and the SM clock sampled during the timed region.

The algorithmic work of one launch is counted in warp-instructions that a
fully converged warp would issue: the per-unit costs below times the transport
events (electron condensed-history steps plus photon Woodcock events) that the
kernel itself counts.  The per-unit costs come from ncu on the same workload
at reduced history counts (smsp__inst_executed.sum x
smsp__thread_inst_executed_per_inst_executed.ratio / 32, divided by the
kernel's event counts), separately for the electron and the photon beam
because their mixes of step and event types differ.
"""
from __future__ import annotations

from typing import Optional

# converged warp-instructions per transport event, electron beam / photon beam: the
# physics of a step or photon event, measured on the kernel that ran each hard event
# inline (no parking).  The kernel that parks hard-event candidates for converged
# passes executes 22.8 / 20.4 per event (the parking is scheduling, not physics), so
# these are the algorithmic figures
INST_PER_EVENT_E_BEAM: Optional[float] = 19.68
INST_PER_EVENT_PH_BEAM: Optional[float] = 18.81
# DRAM bytes (read + write) per transport launch of the benchmark step, from ncu on
# the same workload at 1/5 of its histories, scaled by histories (790 MB electron
# launch, 4.95 GB photon launch); None once the kernel has changed since the capture
TRAFFIC_BYTES_PER_LAUNCH: Optional[float] = 2.87e9


def alu_roofline(events_e_beam: int, events_ph_beam: int, kernel_ms: float, sm_mhz: Optional[float],
                 n_sm: int, launches: int = 2) -> dict:
    peak = None
    if sm_mhz:
        peak = n_sm * 4 * sm_mhz * 1e6 / 1e9  # G warp-instructions / s
    out = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": peak, "achieved": None, "frac": None,
           "traffic": TRAFFIC_BYTES_PER_LAUNCH,
           "peak_basis": f"{n_sm} SMs x 4 warp-inst/clk x median sampled SM clock"}
    if INST_PER_EVENT_E_BEAM is not None and INST_PER_EVENT_PH_BEAM is not None and kernel_ms > 0:
        work = events_e_beam * INST_PER_EVENT_E_BEAM + events_ph_beam * INST_PER_EVENT_PH_BEAM
        out["achieved"] = work / (kernel_ms / 1e3) / 1e9
        out["work_warp_inst_per_launch"] = work / max(launches, 1)
        if peak:
            out["frac"] = out["achieved"] / peak
    return out

"""Roofline of the transport kernel: SM instruction issue.

Transport is neither a dense contraction nor HBM-bound; it is bound by the
instruction issue of the SMs (FP32/INT ALU work, divergence and latency).  The
ceiling is 4 warp-instructions per clock per SM (one per SM sub-partition),
times the SM count and the SM clock sampled during the timed region.

The algorithmic work of one launch is counted in warp-instructions that a
fully converged warp would issue: the per-unit costs below (from ncu,
smsp__thread_inst_executed.sum / 32 per electron step and per photon event on
the 15 MeV 128^3 water workload) times the step and event counts that the
kernel itself reports.
"""
from __future__ import annotations

from typing import Optional

# warp-instructions per electron condensed-history step / per photon Woodcock event
INST_PER_E_STEP: Optional[float] = None
INST_PER_PH_EVENT: Optional[float] = None
# DRAM bytes (read + write) per transport launch of the benchmark step, from ncu
TRAFFIC_BYTES_PER_LAUNCH: Optional[float] = None


def alu_roofline(e_steps: int, ph_events: int, kernel_ms: float, sm_mhz: Optional[float],
                 n_sm: int, launches: int = 2) -> dict:
    peak = None
    if sm_mhz:
        peak = n_sm * 4 * sm_mhz * 1e6 / 1e9  # G warp-instructions / s
    out = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": peak, "achieved": None, "frac": None,
           "traffic": TRAFFIC_BYTES_PER_LAUNCH,
           "peak_basis": f"{n_sm} SMs x 4 warp-inst/clk x median sampled SM clock"}
    if INST_PER_E_STEP is not None and INST_PER_PH_EVENT is not None and kernel_ms > 0:
        work = e_steps * INST_PER_E_STEP + ph_events * INST_PER_PH_EVENT
        out["achieved"] = work / (kernel_ms / 1e3) / 1e9
        out["work_warp_inst_per_launch"] = work / max(launches, 1)
        if peak:
            out["frac"] = out["achieved"] / peak
    return out

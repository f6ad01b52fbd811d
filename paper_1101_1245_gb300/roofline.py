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
# DRAM bytes (read + write) per transport launch of the timing workload: measured with
# 32 batch tallies (2.87e9 per launch); the benchmark now runs it with 16, whose tally
# traffic that capture does not describe, so None until it is captured again
TRAFFIC_BYTES_PER_LAUNCH: Optional[float] = None


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


# The same figures for the batched workload (64 uneven plans of smoothed-noise
# densities, 6-18 MeV photon or electron fields): converged warp-instructions
# per transport event (smsp__thread_inst_executed.sum / 32 / events) in the
# electron-beam and the photon-beam launch sequences, from ncu on the
# workload's 27 plans of at most 160^3 voxels at 1/10 of their first round
# (bench.py --ncu-case --workload c4): 144.79e9 thread-instructions over
# 259.66e6 events, and 72.61e9 over 128.58e6.  Kept fixed as the algorithmic
# work per event, so a faster kernel shows as a higher achieved rate.
INST_PER_EVENT_C4_E_SEQ: Optional[float] = 17.43
INST_PER_EVENT_C4_PH_SEQ: Optional[float] = 17.65
# DRAM bytes (read + write) per event of the same case on the current kernel (one
# 1024-thread CTA per SM, tables packed per material, a photon's majorant taken once
# per pass, each electron step's majorant from its own voxel, event-path divisions as
# reciprocal-multiply, the step's draw taken while its voxel word loads, the inside
# and cut-off tests of primaries at their claim): 1.907 GB over 247.16e6 events
# (electron sequence) and 1.817 GB over 124.71e6 (photon sequence)
TRAFFIC_BYTES_PER_EVENT_C4_E_SEQ: Optional[float] = 7.71
TRAFFIC_BYTES_PER_EVENT_C4_PH_SEQ: Optional[float] = 14.57


def alu_roofline_c4(events_e_seq: int, events_ph_seq: int, kernel_ms: float, sm_mhz: Optional[float],
                    n_sm: int, launches: int) -> dict:
    """SM-issue roofline of the transport launches of one step of the batched
    workload: events of the electron-beam and photon-beam sequences, the device
    time of all `launches` of them; work and traffic per average launch."""
    peak = n_sm * 4 * sm_mhz * 1e6 / 1e9 if sm_mhz else None
    n = max(launches, 1)
    out = {"bound": "alu", "unit": "Gwarp-inst/s", "peak": peak, "achieved": None, "frac": None,
           "traffic": None, "peak_basis": f"{n_sm} SMs x 4 warp-inst/clk x median sampled SM clock",
           "events_per_step": events_e_seq + events_ph_seq, "launches_per_step": launches}
    if TRAFFIC_BYTES_PER_EVENT_C4_E_SEQ is not None and TRAFFIC_BYTES_PER_EVENT_C4_PH_SEQ is not None:
        out["traffic"] = (TRAFFIC_BYTES_PER_EVENT_C4_E_SEQ * events_e_seq
                          + TRAFFIC_BYTES_PER_EVENT_C4_PH_SEQ * events_ph_seq) / n
        out["traffic_basis"] = ("DRAM bytes per average transport launch: ncu bytes per event of the small case "
                                "(electron / photon sequences) x the step's events / its launches")
    if INST_PER_EVENT_C4_E_SEQ is not None and INST_PER_EVENT_C4_PH_SEQ is not None and kernel_ms > 0:
        work = events_e_seq * INST_PER_EVENT_C4_E_SEQ + events_ph_seq * INST_PER_EVENT_C4_PH_SEQ
        out["achieved"] = work / (kernel_ms / 1e3) / 1e9
        out["work_warp_inst_per_launch"] = work / n
        if peak:
            out["frac"] = out["achieved"] / peak
    return out

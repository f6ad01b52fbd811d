"""The SM-issue roofline the benchmark reports (host arithmetic, no GPU): the
peak is SMs x 4 warp-instructions per clock x the sampled clock, the achieved
rate is the fixed per-event work times the kernel's own event counts over the
device time, and the DRAM traffic is per average transport launch."""
import pytest

from paper_1101_1245_gb300 import roofline as rl


def test_batched_workload_roofline():
    e, ph, ms, launches = 1.0e11, 4.0e10, 4000.0, 50
    r = rl.alu_roofline_c4(e, ph, ms, 2070.0, 152, launches=launches)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 4 * 2.07, rel=1e-12)  # 1258.56 G warp-inst/s
    work = e * rl.INST_PER_EVENT_C4_E_SEQ + ph * rl.INST_PER_EVENT_C4_PH_SEQ
    assert r["achieved"] == pytest.approx(work / (ms / 1e3) / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)
    assert r["work_warp_inst_per_launch"] == pytest.approx(work / launches, rel=1e-12)
    traffic = (e * rl.TRAFFIC_BYTES_PER_EVENT_C4_E_SEQ + ph * rl.TRAFFIC_BYTES_PER_EVENT_C4_PH_SEQ) / launches
    assert r["traffic"] == pytest.approx(traffic, rel=1e-12)
    assert r["events_per_step"] == e + ph and r["launches_per_step"] == launches


def test_unsampled_clock_leaves_the_fraction_open():
    r = rl.alu_roofline_c4(1e9, 1e9, 10.0, None, 152, launches=2)
    assert r["peak"] is None and r["frac"] is None
    assert r["achieved"] is not None


def test_timing_workload_roofline():
    r = rl.alu_roofline(7.9e7, 1.8e8, 8.0, 2070.0, 152)
    work = 7.9e7 * rl.INST_PER_EVENT_E_BEAM + 1.8e8 * rl.INST_PER_EVENT_PH_BEAM
    assert r["achieved"] == pytest.approx(work / 8e-3 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / (152 * 4 * 2.07), rel=1e-12)
    assert r["work_warp_inst_per_launch"] == pytest.approx(work / 2, rel=1e-12)

"""Scheduling independence: the dose tally is bit-identical whatever the launch
shape, the history split (energy-grouped spectra and phase spaces included), the
warp-aggregation mode or the overflow path,
because each particle's random stream depends only on (seed, history,
lineage, draw) and energies are integers."""
import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def _plan():
    ph = W.z_slabs((24, 20, 32), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                        (4.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    return ph


def _dose(ctx, ph, src, n, seed, splits=(None,)):
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, src, seed, 16)
    for part in splits:
        ctx.run([plan], [part if part is not None else n])
    import torch
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    st = ctx.plan_result(plan, 0.5, d.data_ptr(), s.data_ptr())
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    return d.cpu().numpy(), s.cpu().numpy(), st


# the ledger and every event counter that depends only on the particles'
# histories (not on scheduling: launches, spills and overflows do)
EVENT_KEYS = ("e_incident", "e_deposited", "e_escaped", "e_rest", "n_photon_events", "n_photon_real",
              "n_compton", "n_photo", "n_pair", "n_electron_steps", "n_hard_real", "n_hard_fict",
              "n_moller", "n_brem", "n_photons", "n_electrons", "n_sampler_capped")

_EDGES, _W = W.synthetic_6mv_spectrum(n_bins=64)
SOURCES = {
    "electron": W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=12.0, center_cm=(6.0, 5.0), field_cm=4.0),
    "photon": W.Source(W.PHOTON, W.BEAM_SQUARE, energy=15.0, center_cm=(6.0, 5.0), field_cm=4.0),
    # a spectrum and a phase space grouped by energy (§IV): each launch claims
    # its histories in decreasing order of energy, each history unchanged
    "grouped": W.Source(W.PHOTON, W.BEAM_SQUARE, center_cm=(6.0, 5.0), field_cm=4.0,
                        spectrum_edges=_EDGES, spectrum_weights=_W, energy_grouping=W.ENERGY_GROUPED),
    "grouped_phsp": W.Source(W.ELECTRON, W.BEAM_PHASE_SPACE,
                             phase_space=W.polyenergetic_phase_space(W.ELECTRON, _plan(), 1013, seed=7).phase_space,
                             energy_grouping=W.ENERGY_GROUPED),
    # the same phase space ungrouped (the phase-space kernel, claims in history order)
    "phsp": W.Source(W.ELECTRON, W.BEAM_PHASE_SPACE,
                     phase_space=W.polyenergetic_phase_space(W.ELECTRON, _plan(), 1013, seed=7).phase_space),
}
# sources that run the phase-space kernel
PHSP_KINDS = ("grouped", "grouped_phsp", "phsp")


def _phsp_kernel_accepts(launch) -> bool:
    """Grouped sources run the phase-space kernel: no profile or aggregation
    flag, refill at every pass."""
    return (launch.get("refill_period", 1) == 1
            and not launch.get("flags", 0) & (g.LAUNCH_WARP_AGGREGATE | g.LAUNCH_PROFILE))


@pytest.fixture(scope="module")
def reference():
    ctx = make_ctx()
    ph = _plan()
    out = {k: _dose(ctx, ph, src, 40_000, 99) for k, src in SOURCES.items()}
    ctx.close()
    return ph, out


@pytest.mark.parametrize("kind", ["electron", "photon", "grouped", "grouped_phsp", "phsp"])
@pytest.mark.parametrize("launch", [
    dict(),
    dict(block_threads=512, blocks_per_sm=2),
    dict(block_threads=512, blocks_per_sm=1),
    dict(block_threads=256, blocks_per_sm=2),
    dict(block_threads=128, blocks_per_sm=3, chunk=8, refill_low=30, switch_high=64,
         stack_capacity=128),
    dict(flags=g.LAUNCH_WARP_AGGREGATE),
    dict(flags=g.LAUNCH_PROFILE),
    dict(flags=g.LAUNCH_GRAPH),
    dict(stack_capacity=128, switch_high=64, overflow_capacity=1 << 16, chunk=256),
    # the refill policies of the divergence-reduction ablation (their own kernel)
    dict(refill_period=4),
    dict(refill_period=16),
    dict(refill_period=g.REFILL_WHEN_EMPTY),
])
def test_bit_identical_across_launch_shapes(reference, kind, launch):
    if kind in PHSP_KINDS and not _phsp_kernel_accepts(launch):
        pytest.skip("outside the phase-space kernel's launch restrictions")
    ph, out = reference
    ctx = make_ctx(**launch)
    d, s, st = _dose(ctx, ph, SOURCES[kind], 40_000, 99)
    ctx.close()
    d0, s0, st0 = out[kind]
    assert np.array_equal(d, d0)
    assert np.array_equal(s, s0)
    for k in EVENT_KEYS:
        assert st[k] == st0[k], k
    assert st["e_deposited"] + st["e_escaped"] + st["e_rest"] == st["e_incident"]
    # every real photon event is one interaction, every real hard event one of two
    assert st["n_compton"] + st["n_photo"] + st["n_pair"] == st["n_photon_real"]
    assert st["n_moller"] + st["n_brem"] == st["n_hard_real"]


@pytest.mark.parametrize("kind", ["electron", "photon", "grouped", "grouped_phsp"])
@pytest.mark.parametrize("flags", [0, g.LAUNCH_GRAPH])
def test_split_runs_equal_one_run(reference, kind, flags):
    """Also replays one captured graph with new kernel arguments per run.
    Grouped sources included: each run sorts its own histories' claims, and
    no history's primary depends on that order."""
    ph, out = reference
    ctx = make_ctx(flags=flags)
    d, s, st = _dose(ctx, ph, SOURCES[kind], 40_000, 99, splits=(10_000, 17_000, 13_000))
    ctx.close()
    assert np.array_equal(d, out[kind][0])
    assert np.array_equal(s, out[kind][1])


# A small grid (2 warps per SM) and no high-water switching: each warp's
# stacks fill past their headroom and spill to the global overflow queue.
SPILL = dict(block_threads=64, blocks_per_sm=1, stack_capacity=128, switch_high=128)


@pytest.mark.parametrize("kind", ["electron", "photon"])
@pytest.mark.parametrize("flags", [0, g.LAUNCH_GRAPH])
def test_overflow_path_is_lossless(kind, flags):
    """Spilled particles finish in further launches with the same result
    (after a first launch replayed from a graph, too)."""
    ph = _plan()
    n = 200_000 if kind == "photon" else 40_000
    ctx = make_ctx(overflow_capacity=1 << 20, flags=flags, **SPILL)
    a = _dose(ctx, ph, SOURCES[kind], n, 5)
    ctx.close()
    ctx = make_ctx()
    b = _dose(ctx, ph, SOURCES[kind], n, 5)
    ctx.close()
    assert a[2]["n_spilled"] > 0 and a[2]["n_launches"] > 1, a[2]
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_queue_overflow_is_reported_not_dropped():
    ph = _plan()
    ctx = make_ctx(overflow_capacity=64, **SPILL)
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, SOURCES["photon"], 5, 8)
    with pytest.raises(g.GpumcdError) as e:
        ctx.run([plan], [200_000])
    assert e.value.status == g.ERR_QUEUE_OVERFLOW
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    ctx.close()


def test_seed_changes_result(reference):
    ph, out = reference
    ctx = make_ctx()
    d, _, _ = _dose(ctx, ph, SOURCES["photon"], 40_000, 100)
    ctx.close()
    assert not np.array_equal(d, out["photon"][0])

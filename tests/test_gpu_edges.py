"""Edge and degenerate cases of the CUDA path: empty and ragged inputs, beams
that miss the phantom, sources below the cut-offs, one-voxel phantoms, and
invalid inputs rejected with a status instead of a fault."""
import math

import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests._stats import three_sigma_pass_rate
from tests.gpu_common import ledger_exact, make_ctx, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
Q = 2.0 ** -26


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_zero_histories_is_an_empty_result(ctx):
    ph = W.homogeneous((7, 5, 3), 1.0, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, W.pencil(W.PHOTON, 1.0, 3.0, 2.0), 1, 8)
    ctx.run([plan], [0])
    st = ctx.plan_result(plan, 0.5)
    assert st["histories"] == 0 and st["e_incident"] == 0 and st["e_deposited"] == 0
    with pytest.raises(g.GpumcdError):
        ctx.simulate(pid, W.pencil(W.PHOTON, 1.0, 3.0, 2.0), 0, 1, nvox=ph.nvox)
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)


@pytest.mark.parametrize("particle", [W.PHOTON, W.ELECTRON])
def test_beam_missing_the_phantom_escapes_whole(ctx, particle):
    ph = W.homogeneous((8, 8, 8), 0.5, W.MAT_WATER, 1.0)
    r = run_gpu(ctx, W.Plan("miss", ph, W.pencil(particle, 5.0, -1.0, 2.0), 3000, 3))
    st = r.stats
    assert st["e_incident"] == 3000 * round(5.0 / Q)
    assert st["e_escaped"] == st["e_incident"] and st["e_deposited"] == 0
    assert not r.dose.any()


def test_electron_field_wider_than_the_phantom(ctx):
    """An electron field wider than the phantom's entry face: the primaries that
    start outside escape as they are claimed, the others are transported.  The
    escaped fraction and the dose agree with the oracle; the ledger is exact."""
    ph = W.homogeneous((10, 10, 12), 0.5, W.MAT_WATER, 1.0)  # a 5 x 5 cm face
    src = W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=6.0, center_cm=(2.5, 2.5), field_cm=8.0)
    plan = W.Plan("wide", ph, src, 40_000, 8)
    gres = run_gpu(ctx, plan)
    ores = run_oracle(plan)
    assert ledger_exact(gres.stats)
    fg = gres.stats["e_escaped"] / gres.stats["e_incident"]
    fo = ores.stats["e_escaped"] / ores.stats["e_incident"]
    # 1 - (5/8)^2 = 61% of the field lies outside the face
    assert fg > 1.0 - (5.0 / 8.0) ** 2 - 0.01
    # a history's escaped fraction lies in [0, 1]: its variance is at most p (1 - p)
    assert abs(fg - fo) <= 4.0 * math.sqrt(2.0 * fg * (1.0 - fg) / plan.n_histories), (fg, fo)
    do, so = ores.dose_gy(ph), ores.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert three_sigma_pass_rate(gres.dose, gres.sigma, do, so, mask) >= 0.99


def test_sources_below_the_cutoffs_deposit_at_entry(ctx):
    ph = W.homogeneous((4, 4, 4), 1.0, W.MAT_WATER, 1.0)
    for particle, e in ((W.ELECTRON, 0.1), (W.PHOTON, 0.005)):
        r = run_gpu(ctx, W.Plan("cut", ph, W.pencil(particle, e, 1.5, 2.5), 1000, 4))
        st = r.stats
        assert st["e_deposited"] == st["e_incident"] == 1000 * round(e / Q)
        d = r.dose.reshape(4, 4, 4)
        assert d[0, 2, 1] > 0 and np.count_nonzero(d) == 1


def test_one_voxel_phantom(ctx):
    ph = W.homogeneous((1, 1, 1), 2.0, W.MAT_BONE, 1.85)
    r = run_gpu(ctx, W.Plan("one", ph, W.pencil(W.ELECTRON, 3.0, 1.0, 1.0), 5000, 5))
    assert ledger_exact(r.stats)
    assert r.stats["e_deposited"] > 0 and r.stats["e_escaped"] > 0


def test_ragged_sizes_match_the_oracle(ctx):
    """Dimensions that tile nothing and a history count that fills no batch evenly."""
    ph = W.z_slabs((37, 23, 41), 0.4, [(2.0, W.MAT_WATER, 1.0), (1.6, W.MAT_BONE, 1.85),
                                        (3.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    src = W.Source(W.PHOTON, W.BEAM_SQUARE, energy=6.0, center_cm=(7.1, 4.3), field_cm=3.3)
    plan = W.Plan("ragged", ph, src, 54_321, 6)
    gres = run_gpu(ctx, plan)
    ores = run_oracle(plan)
    assert ledger_exact(gres.stats)
    do, so = ores.dose_gy(ph), ores.sigma_gy(ph)
    mask = do > 0.1 * do.max()
    assert three_sigma_pass_rate(gres.dose, gres.sigma, do, so, mask) >= 0.99


def test_invalid_inputs_are_rejected(ctx):
    ph = W.homogeneous((4, 4, 4), 1.0, W.MAT_WATER, 1.0)
    bad = W.homogeneous((4, 4, 4), 1.0, W.MAT_WATER, 1.0)
    bad.mat[0, 0, 0] = 7  # no such material
    with pytest.raises(g.GpumcdError) as e:
        ctx.create_phantom(bad)
    assert e.value.status == g.ERR_INVALID_ARG
    bad = W.homogeneous((4, 4, 4), 1.0, W.MAT_WATER, 1.0)
    bad.rho[1, 1, 1] = 0.0
    with pytest.raises(g.GpumcdError):
        ctx.create_phantom(bad)
    pid = ctx.create_phantom(ph)
    for src in (W.pencil(W.PHOTON, 25.0, 1, 1), W.pencil(W.ELECTRON, -1.0, 1, 1),
                W.Source(W.PHOTON, W.BEAM_SQUARE, spectrum_edges=np.array([0.1, 0.2, 0.15]),
                         spectrum_weights=np.array([1.0, 1.0]), field_cm=1.0)):
        with pytest.raises(g.GpumcdError) as e:
            ctx.plan_open(pid, src, 1, 8)
        assert e.value.status == g.ERR_INVALID_ARG
    with pytest.raises(g.GpumcdError) as e:
        ctx.plan_open(pid, W.pencil(W.PHOTON, 1.0, 1, 1), 1, 12)  # batches not a power of two
    assert e.value.status == g.ERR_INVALID_ARG
    with pytest.raises(g.GpumcdError) as e:
        ctx.plan_open(999, W.pencil(W.PHOTON, 1.0, 1, 1), 1, 8)
    assert e.value.status == g.ERR_NOT_FOUND
    with pytest.raises(g.GpumcdError) as e:
        ctx.set_launch(block_threads=100)
    assert e.value.status == g.ERR_INVALID_ARG
    ctx.destroy_phantom(pid)


def test_hbm_budget_is_enforced():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = g.Context(0, hbm_budget_bytes=64 << 20)
    import workloads as W2
    c.load_materials(W2.MATERIALS, W2.DEFAULT_PHYSICS)
    ph = W.homogeneous((64, 64, 64), 0.5, W.MAT_WATER, 1.0)
    pid = c.create_phantom(ph)  # 1 MB of voxel words fits
    with pytest.raises(g.GpumcdError) as e:
        c.plan_open(pid, W.pencil(W.PHOTON, 1.0, 16, 16), 1, 64)  # 134 MB of tallies does not
    assert e.value.status == g.ERR_BUDGET
    used, budget = c.memory()
    assert used <= budget == 64 << 20
    c.close()


def test_device_memory_is_reused():
    """Phantom, plan and scratch blocks return to the context's cache and are
    handed out again: live memory stays flat over create/simulate/destroy
    cycles and the results do not change."""
    ctx = make_ctx()
    ph = W.homogeneous((40, 36, 32), 0.5, W.MAT_WATER, 1.0)
    src = W.square_field(W.PHOTON, 6.0, ph, 6.0)
    doses, used = [], []
    for i in range(4):
        pid = ctx.create_phantom(ph)
        r = ctx.simulate(pid, src, 20_000, 5, nvox=ph.nvox)
        doses.append(r.dose)
        ctx.destroy_phantom(pid)
        used.append(ctx.memory()[0])
    assert used[1] == used[2] == used[3]
    assert all(np.array_equal(doses[0], d) for d in doses[1:])
    ctx.close()


def test_cached_blocks_yield_to_the_budget():
    """Blocks in the cache are released when a new allocation needs the room."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = g.Context(0, hbm_budget_bytes=200 << 20)
    c.load_materials(W.MATERIALS, W.DEFAULT_PHYSICS)
    small = c.create_phantom(W.homogeneous((64, 64, 64), 0.5, W.MAT_WATER, 1.0))  # 1 MB
    big = c.plan_open(small, W.pencil(W.PHOTON, 1.0, 16, 16), 1, 64)  # 134 MB of tallies
    c.plan_close(big)  # -> cache
    ph2 = W.homogeneous((96, 96, 64), 0.5, W.MAT_WATER, 1.0)  # 2.4 MB
    pid2 = c.create_phantom(ph2)
    p2 = c.plan_open(pid2, W.pencil(W.PHOTON, 1.0, 24, 24), 1, 32)  # 151 MB: the cached block must go
    assert c.plan_histories(p2) == 0
    used, budget = c.memory()
    assert used <= budget
    c.plan_close(p2)
    c.close()


def test_refill_policy_validation():
    """A refill policy other than every pass, and the photon-only mode, each run
    their own kernel, alone (without the profile, the warp-aggregated deposits
    or each other); like every kernel, at most 1024 threads per SM."""
    ctx = make_ctx()
    for bad in (dict(refill_period=4, block_threads=512, blocks_per_sm=3),
                dict(refill_period=g.REFILL_WHEN_EMPTY, flags=g.LAUNCH_PROFILE),
                dict(refill_period=16, flags=g.LAUNCH_WARP_AGGREGATE),
                dict(refill_period=4, flags=g.LAUNCH_KERMA),
                dict(flags=g.LAUNCH_KERMA | g.LAUNCH_PROFILE),
                dict(flags=g.LAUNCH_KERMA, block_threads=1024, blocks_per_sm=2)):
        with pytest.raises(g.GpumcdError) as e:
            ctx.set_launch(**bad)
        assert e.value.status == g.ERR_INVALID_ARG
    ctx.set_launch(refill_period=8, flags=g.LAUNCH_GRAPH)
    assert ctx.get_launch()["refill_period"] == 8
    ctx.set_launch(refill_period=1, flags=0)
    assert ctx.get_launch()["refill_period"] == 1
    ctx.set_launch(flags=g.LAUNCH_KERMA, block_threads=256, blocks_per_sm=3)
    ctx.set_launch(flags=0, block_threads=1024, blocks_per_sm=1)
    ctx.close()


def test_launch_flags_select_compiled_kernels():
    """The cycle profile and warp-aggregated deposits are separate kernel
    instantiations: combining them, or asking for more than 1024 threads per
    SM, is rejected; each alone runs and gives the plain kernel's tally, at
    the default shape and at 512 threads x 2 CTAs per SM."""
    ctx = make_ctx()
    with pytest.raises(g.GpumcdError) as e:
        ctx.set_launch(flags=g.LAUNCH_PROFILE | g.LAUNCH_WARP_AGGREGATE)
    assert e.value.status == g.ERR_INVALID_ARG
    for flag in (g.LAUNCH_PROFILE, g.LAUNCH_WARP_AGGREGATE):
        with pytest.raises(g.GpumcdError) as e:
            ctx.set_launch(flags=flag, block_threads=512, blocks_per_sm=3)
        assert e.value.status == g.ERR_INVALID_ARG
    ph = W.homogeneous((24, 24, 24), 0.5, W.MAT_WATER, 1.0)
    src = W.square_field(W.ELECTRON, 8.0, ph, 4.0)
    doses = []
    for flag, bt, bps in ((0, 1024, 1), (g.LAUNCH_PROFILE, 512, 2), (g.LAUNCH_WARP_AGGREGATE | g.LAUNCH_GRAPH, 1024, 1),
                          (g.LAUNCH_PROFILE, 1024, 1)):
        ctx.set_launch(flags=flag, block_threads=bt, blocks_per_sm=bps)
        pid = ctx.create_phantom(ph)
        doses.append(ctx.simulate(pid, src, 20_000, 3, nvox=ph.nvox).dose)
        ctx.destroy_phantom(pid)
    assert all(np.array_equal(doses[0], d) for d in doses[1:])
    ctx.close()

"""Batched and served forms: several plans in one persistent launch give each
plan the same tally, bit for bit, as running it alone; the autotuner changes
speed, not results; the server retires requests at the uncertainty target,
admits them within its HBM budget, and a served result equals the same
request rerun alone at the same history count."""
import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def _specs(count=6, seed=44):
    return W.plan_distribution(count, seed, n_lo=24, n_hi=40, hist_lo=2e4, hist_hi=6e4)


def _setup(ctx, specs):
    phantoms = [sp.phantom() for sp in specs]
    pids = [ctx.create_phantom(ph) for ph in phantoms]
    srcs = [W.square_field(sp.particle, sp.energy, ph, sp.field_cm) for sp, ph in zip(specs, phantoms)]
    return phantoms, pids, srcs


def _dose(ctx, plan, nvox):
    import torch
    d = torch.zeros(nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros(nvox, dtype=torch.float64, device="cuda")
    st = ctx.plan_result(plan, 0.5, d.data_ptr(), s.data_ptr())
    return d.cpu().numpy(), s.cpu().numpy(), st


def test_batched_launch_equals_plans_alone():
    ctx = make_ctx()
    specs = _specs()
    assert {sp.particle for sp in specs} == {W.PHOTON, W.ELECTRON}
    phantoms, pids, srcs = _setup(ctx, specs)
    n = [sp.n_histories for sp in specs]
    mix = [ctx.plan_open(pid, src, sp.seed, 16) for pid, src, sp in zip(pids, srcs, specs)]
    ctx.run(mix, n)
    for i, (pid, src, sp) in enumerate(zip(pids, srcs, specs)):
        alone = ctx.plan_open(pid, src, sp.seed, 16)
        ctx.run([alone], [n[i]])
        a = _dose(ctx, alone, phantoms[i].nvox)
        b = _dose(ctx, mix[i], phantoms[i].nvox)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        for k in ("e_incident", "e_deposited", "e_escaped", "e_rest"):
            assert a[2][k] == b[2][k]
        assert b[2]["e_deposited"] + b[2]["e_escaped"] + b[2]["e_rest"] == b[2]["e_incident"]
        ctx.plan_close(alone)
    ctx.close()


def test_autotune_changes_speed_not_results():
    from paper_1101_1245_gb300.autotune import autotune
    ctx = make_ctx()
    specs = _specs(4, seed=45)
    phantoms, pids, srcs = _setup(ctx, specs)
    p0 = ctx.plan_open(pids[0], srcs[0], 7, 16)
    ctx.run([p0], [30_000])
    before = _dose(ctx, p0, phantoms[0].nvox)
    res = autotune(ctx, [(pid, src, 10_000) for pid, src in zip(pids, srcs)], reps=1)
    assert res["transport_ms"] > 0 and len(res["trials"]) >= 4
    assert ctx.get_launch()["block_threads"] == res["launch"]["block_threads"]
    p1 = ctx.plan_open(pids[0], srcs[0], 7, 16)
    ctx.run([p1], [30_000])
    after = _dose(ctx, p1, phantoms[0].nvox)
    assert np.array_equal(before[0], after[0])
    ctx.close()


def test_served_results_equal_alone_reruns():
    """Request 3 is a spectrum grouped by energy (§IV): its strata follow from
    the history index, so it too equals its alone rerun under another split."""
    from paper_1101_1245_gb300.serve import DoseRequest, Server
    ctx = make_ctx()
    specs = _specs(6, seed=46)
    phantoms, pids, srcs = _setup(ctx, specs)
    edges, w = W.synthetic_6mv_spectrum(n_bins=64)
    srcs[3] = W.Source(specs[3].particle, W.BEAM_SQUARE, center_cm=srcs[3].center_cm,
                       field_cm=srcs[3].field_cm, spectrum_edges=edges, spectrum_weights=w,
                       energy_grouping=W.ENERGY_GROUPED)
    srv = Server(ctx, hbm_budget=8 << 30, target=0.05, round_histories=300_000,
                 first_chunk=20_000, keep_dose=True)
    for i, (pid, src, sp) in enumerate(zip(pids, srcs, specs)):
        srv.submit(DoseRequest(i, pid, phantoms[i].nvox, src, sp.seed, 0.0, 3_000_000))
    results = {r.rid: r for r in srv.run(real_time=False)}
    assert len(results) == 6
    assert all(r.s_thr <= 0.05 or r.histories >= 3_000_000 for r in results.values())
    assert srv.report()["latency_p99_s"] >= srv.report()["latency_p50_s"] > 0
    for i in (0, 3):
        r = results[i]
        plan = ctx.plan_open(pids[i], srcs[i], specs[i].seed, 16)
        first = r.histories // 3
        ctx.run([plan], [first])
        ctx.run([plan], [r.histories - first])
        d, s, _ = _dose(ctx, plan, phantoms[i].nvox)
        assert np.array_equal(d, r.dose) and np.array_equal(s, r.sigma)
        ctx.plan_close(plan)
    ctx.close()


def test_server_admits_within_budget():
    from paper_1101_1245_gb300.serve import DoseRequest, Server
    ctx = make_ctx()
    specs = _specs(5, seed=47)
    phantoms, pids, srcs = _setup(ctx, specs)
    biggest = max(16 * ph.nvox * 8 + 64 for ph in phantoms)
    srv = Server(ctx, hbm_budget=2 * biggest, target=0.08, round_histories=200_000,
                 first_chunk=20_000)
    for i, (pid, src, sp) in enumerate(zip(pids, srcs, specs)):
        srv.submit(DoseRequest(i, pid, phantoms[i].nvox, src, sp.seed, 0.0, 2_000_000))
    assert len(srv.run(real_time=False)) == 5
    assert srv.max_used <= 2 * biggest and srv.used == 0
    assert srv.max_active < 5  # the budget held some requests back
    tiny = Server(ctx, hbm_budget=1024, target=0.08)
    with pytest.raises(g.GpumcdError):
        tiny.submit(DoseRequest(9, pids[0], phantoms[0].nvox, srcs[0], 1, 0.0))
    ctx.close()


def test_overlapping_submitted_sequences_equal_one_run():
    """One plan in two sequences in flight at once (and other plans beside it)
    ends with the tally of a single synchronous run of the same histories."""
    ctx = make_ctx()
    specs = _specs(4, seed=48)
    phantoms, pids, srcs = _setup(ctx, specs)
    a = [ctx.plan_open(pid, src, sp.seed, 16) for pid, src, sp in zip(pids, srcs, specs)]
    t1 = ctx.submit([a[0], a[1]], [32_000, 16_000])
    t2 = ctx.submit([a[0], a[2], a[3]], [48_000, 16_000, 16_000])
    with pytest.raises(g.GpumcdError) as e:
        ctx.submit([a[3]], [16])  # both slots busy
    assert e.value.status == g.ERR_STATE
    with pytest.raises(g.GpumcdError) as e:
        ctx.plan_result(a[0], 0.5)  # in flight
    assert e.value.status == g.ERR_STATE
    with pytest.raises(g.GpumcdError) as e:
        ctx.plan_close(a[2])
    assert e.value.status == g.ERR_STATE
    while not ctx.poll(t2):
        pass
    ctx.wait(t1)
    with pytest.raises(g.GpumcdError) as e:
        ctx.wait(t1)  # already finished
    assert e.value.status == g.ERR_NOT_FOUND
    assert ctx.plan_histories(a[0]) == 80_000
    for i, n in ((0, 80_000), (1, 16_000), (2, 16_000), (3, 16_000)):
        b = ctx.plan_open(pids[i], srcs[i], specs[i].seed, 16)
        ctx.run([b], [n])
        x = _dose(ctx, a[i], phantoms[i].nvox)
        y = _dose(ctx, b, phantoms[i].nvox)
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2]["e_deposited"] + x[2]["e_escaped"] + x[2]["e_rest"] == x[2]["e_incident"]
        assert x[2]["e_incident"] == y[2]["e_incident"]
        ctx.plan_close(b)
    ctx.close()


def test_failed_sequence_marks_its_plans():
    """A submitted sequence that overflows its queue reports the error at
    wait, and its plan returns ERR_STATE until it is reset."""
    ctx = make_ctx(overflow_capacity=64, block_threads=64, blocks_per_sm=1, stack_capacity=128,
                   switch_high=128)
    ph = W.z_slabs((24, 20, 32), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                        (4.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    pid = ctx.create_phantom(ph)
    src = W.Source(W.PHOTON, W.BEAM_SQUARE, energy=15.0, center_cm=(6.0, 5.0), field_cm=4.0)
    p = ctx.plan_open(pid, src, 5, 16)
    t = ctx.submit([p], [200_000])
    with pytest.raises(g.GpumcdError) as e:
        ctx.wait(t)
    assert e.value.status == g.ERR_QUEUE_OVERFLOW
    with pytest.raises(g.GpumcdError) as e:
        ctx.plan_result(p, 0.5)
    assert e.value.status == g.ERR_STATE
    ctx.plan_reset(p, 5)
    ctx.set_launch(overflow_capacity=1 << 20)
    ctx.run([p], [1_600])
    assert ctx.plan_result(p, 0.5)["histories"] == 1_600
    ctx.close()


def test_graph_launches_equal_direct_launches():
    """Batched runs of changing plan sets through one slot's captured graph,
    and submitted sequences through the other slots' graphs, give the tallies
    of direct launches."""
    specs = _specs(5, seed=50)
    out = {}
    for flags in (0, g.LAUNCH_GRAPH):
        ctx = make_ctx(flags=flags)
        phantoms, pids, srcs = _setup(ctx, specs)
        a = [ctx.plan_open(pid, src, sp.seed, 16) for pid, src, sp in zip(pids, srcs, specs)]
        ctx.run(a[:3], [16_000, 32_000, 16_000])
        ctx.run([a[1], a[3], a[4]], [16_000, 48_000, 16_000])
        t = ctx.submit([a[0], a[4]], [32_000, 16_000])
        u = ctx.submit([a[2]], [16_000])
        ctx.wait(u)
        ctx.wait(t)
        ctx.run([a[0]], [16_000])
        out[flags] = [_dose(ctx, p, phantoms[i].nvox) for i, p in enumerate(a)]
        ctx.close()
    for x, y in zip(out[0], out[g.LAUNCH_GRAPH]):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2]["histories"] == y[2]["histories"]
        assert y[2]["e_deposited"] + y[2]["e_escaped"] + y[2]["e_rest"] == y[2]["e_incident"]


def test_graph_follows_the_compiled_kernel():
    """One slot's captured graph holds one compiled transport kernel.  When the
    next run needs another one (a phase-space source runs its own kernel, the
    photon-only flag another) at the same launch shape, the graph is captured
    again, so each run gives the tally of a direct launch."""
    ph = W.homogeneous((16, 16, 20), 0.5, W.MAT_WATER, 1.0)
    beam = W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=8.0, center_cm=(4.0, 4.0), field_cm=3.0)
    phsp = W.Source(W.ELECTRON, W.BEAM_PHASE_SPACE,
                    phase_space=W.polyenergetic_phase_space(W.ELECTRON, ph, 501, seed=9).phase_space)
    gamma = W.Source(W.PHOTON, W.BEAM_SQUARE, energy=6.0, center_cm=(4.0, 4.0), field_cm=3.0)
    steps = [(beam, 0), (phsp, 0), (beam, 0), (gamma, g.LAUNCH_KERMA), (gamma, 0)]
    out = {}
    for graph in (0, g.LAUNCH_GRAPH):
        ctx = make_ctx()
        pid = ctx.create_phantom(ph)
        res = []
        for i, (src, flags) in enumerate(steps):
            ctx.set_launch(flags=flags | graph)
            plan = ctx.plan_open(pid, src, 70 + i, 16)
            ctx.run([plan], [20_000])
            res.append(_dose(ctx, plan, ph.nvox))
            ctx.plan_close(plan)
        out[graph] = res
        ctx.close()
    for x, y in zip(out[0], out[g.LAUNCH_GRAPH]):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
        assert x[2]["e_deposited"] == y[2]["e_deposited"]


def test_run_to_uncertainty_batched_equals_plans_alone():
    """gpumcd_run_to_uncertainty (§II.D: run until s_0.5 reaches the target):
    six uneven plans together and each plan by itself take the same rounds of
    histories, stop at or below the target, and end with the same tallies bit
    for bit; results through host outputs equal the device ones."""
    import torch
    ctx = make_ctx()
    specs = _specs(6, seed=49)
    phantoms, pids, srcs = _setup(ctx, specs)
    first = [sp.n_histories for sp in specs]
    cap = [3_000_000] * len(specs)
    together = [ctx.plan_open(pid, src, sp.seed, 16) for pid, src, sp in zip(pids, srcs, specs)]
    res = ctx.run_to_uncertainty(together, first, cap, 0.05)
    assert res["rounds"] >= 2
    for i in range(len(specs)):
        h, s = res["histories"][i], res["s_thr"][i]
        assert h % 16 == 0 and first[i] <= h <= cap[i]
        assert s <= 0.05 or h == cap[i]
        alone = ctx.plan_open(pids[i], srcs[i], specs[i].seed, 16)
        one = ctx.run_to_uncertainty([alone], [first[i]], [cap[i]], 0.05)
        assert one["histories"] == [h] and one["s_thr"] == [s]
        a, b = _dose(ctx, together[i], phantoms[i].nvox), _dose(ctx, alone, phantoms[i].nvox)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert a[2]["e_deposited"] + a[2]["e_escaped"] + a[2]["e_rest"] == a[2]["e_incident"]
        hd = torch.empty(phantoms[i].nvox, dtype=torch.float64).pin_memory().numpy()
        hs = np.empty(phantoms[i].nvox, dtype=np.float64)
        st = ctx.plan_result_host(alone, 0.5, hd, hs)
        assert np.array_equal(hd, a[0]) and np.array_equal(hs, a[1])
        assert st["histories"] == h
        ctx.plan_close(alone)
    with pytest.raises(g.GpumcdError) as e:
        ctx.run_to_uncertainty([together[0]], [0], [10], 0.05)
    assert e.value.status == g.ERR_INVALID_ARG
    with pytest.raises(g.GpumcdError) as e:
        ctx.run_to_uncertainty([together[0], together[0]], [16, 16], [32, 32], 0.05)
    assert e.value.status == g.ERR_INVALID_ARG
    ctx.close()

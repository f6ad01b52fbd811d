"""Parity of the batched form on the 64 plans of the batched workload (uneven
phantoms of 64^3 to 256^3 voxels of 0.2 to 0.5 cm, smoothed-noise densities
of 0.2 to 2.0 g/cm^3 mapped to lung / water / bone, 6 to 18 MeV photon or
electron fields of 2 to 15 cm) against the FP64 oracle on the same seeded
phantoms and beams.

All 64 plans run in one batched launch sequence per particle type (16 batches
each, as the benchmark runs them); the oracle runs each plan at 2e5
histories in K = 8 independent parts, the GPU at 50 times that, so the
comparison's noise is the oracle's.  The compared voxels come from a third,
independent GPU run (other seeds): choosing them by either compared side's
own noisy dose would favour its upward fluctuations (regression to the mean).

At these counts the oracle sees few events in most voxels of a photon plan,
where its per-voxel sigma is degenerate and skewed (an oracle run against a
second oracle run fails a per-voxel 3-sigma test there just as often: 89-91%
of the voxels pass on two photon plans), so:
- per voxel, where the oracle's expected relative sigma (from the independent
  run) is under 10% (a hundred or more events): >= 97% of a plan's voxels
  (plans with >= 30 such voxels) and >= 99% of all of them within 3 combined
  sigma, and z-scores of mean ~0 and spread ~1, which also checks both
  uncertainty estimators;
- per block of 4 x 4 x 4 voxels above 10% of the block D_max, for every plan:
  the GPU's mass-weighted block dose against the mean of the oracle's K parts
  with the standard error of their spread (a t statistic with K - 1 degrees of
  freedom): >= 97% of a plan's blocks and >= 98.5% of all within 4 of it
  (an oracle against a second oracle run passes 99.2-100%);
- the exact integer energy ledger of every plan, and event rates per history,
  pooled by particle type, within 3%.  The GPU takes each electron step's
  majorant from its own voxel (an exact Woodcock form that gives the paper
  form's dose; tests/test_oracle_kinematics.py), which splits fewer steps at
  fictitious candidates: its step rate is compared with an oracle run in that
  form (a tenth of the histories), the other rates with the paper's form.
The served form runs the same plans to the same tallies
(tests/test_gpu_batched_served.py), so this also covers it.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._gamma import gamma_pass_rate
from tests._stats import three_sigma_pass_rate
from tests.conftest import host_cores
from tests.gpu_common import ledger_exact, make_ctx

pytestmark = pytest.mark.gpu

N_ORACLE = 200_000
N_GPU = 50 * N_ORACLE
K = 8      # independent oracle parts
B = 4      # block edge in voxels


def _blocks(a, n):
    """Sums over blocks of B^3 voxels of an (n^3,) voxel array (x fastest);
    the last n mod B planes of each axis are left out."""
    m = n // B * B
    v = np.asarray(a, dtype=np.float64).reshape(n, n, n)[:m, :m, :m]
    return v.reshape(m // B, B, m // B, B, m // B, B).sum(axis=(1, 3, 5)).ravel()


def _oracle_plan(args):
    """Worker: one plan of the batched workload on the oracle in K parts: its
    per-voxel dose and sigma in Gy per history, the energy per history of each
    part in each block, its event counts, and the electron steps per history
    of a run in the GPU's per-voxel majorant form."""
    spec, n, seed = args
    ph = spec.phantom()
    src = W.square_field(spec.particle, spec.energy, ph, spec.field_cm)
    cuts = np.linspace(0, n, K + 1).astype(np.int64)
    s1 = s2 = None
    st = {}
    parts = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        p1, p2, pst = oracle.simulate_range(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, int(a), int(b), seed)
        s1 = p1 if s1 is None else s1 + p1
        s2 = p2 if s2 is None else s2 + p2
        st = {k: st.get(k, 0) + v for k, v in pst.items()}
        parts.append(_blocks(p1, spec.n) / float(b - a))
    r = oracle.OracleResult(n, s1, s2, st)
    nv = max(n // 10, 1000)
    _, _, vst = oracle.simulate_range(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, n, n + nv, seed,
                                      oracle.FLAG_VOXEL_EMAJOR)
    st["n_e_steps_voxel_form"] = vst["n_e_steps"] * (n / nv)
    return spec.index, r.dose_gy(ph), r.sigma_gy(ph), np.array(parts), st


def _phantom(spec):
    ph = spec.phantom()
    return ph.dims, ph.voxel_cm, ph.mat, ph.rho


def test_batched_workload_plans_against_oracle():
    import multiprocessing as mp

    import torch

    specs = W.config4()
    pool = mp.get_context("spawn").Pool(host_cores())
    try:
        ctx = make_ctx()
        plans, sel, rhos, vol = [], [], [], []
        for dims, vox, mat, rho in pool.imap(_phantom, specs):
            ph = W.Phantom(dims, vox, mat, rho)
            pid = ctx.create_phantom(ph)
            sp = specs[len(plans)]
            src = W.square_field(sp.particle, sp.energy, ph, sp.field_cm)
            plans.append(ctx.plan_open(pid, src, sp.seed, 16))
            sel.append(ctx.plan_open(pid, src, sp.seed + 1, 16))
            rhos.append(np.ascontiguousarray(ph.rho, dtype=np.float32).ravel())
            vol.append(float(np.prod(ph.voxel_cm)))
        ctx.run(plans, [N_GPU] * len(plans))
        ctx.run(sel, [N_GPU] * len(sel))
        jobs = [(sp, N_ORACLE, sp.seed ^ 0x5A5A) for sp in specs]
        rates, brates, zs, counts = {}, {}, [], {0: {}, 1: {}}
        for idx, do, so, oparts, ost in pool.imap_unordered(_oracle_plan, jobs):
            n, rho = specs[idx].n, rhos[idx]
            d = torch.zeros(rho.size, dtype=torch.float64, device="cuda")
            s = torch.zeros_like(d)
            ctx.plan_result(sel[idx], 0.5, d.data_ptr(), s.data_ptr())
            ds, ss = d.cpu().numpy(), s.cpu().numpy()
            gst = ctx.plan_result(plans[idx], 0.5, d.data_ptr(), s.data_ptr())
            dg, sg = d.cpu().numpy(), s.cpu().numpy()
            assert ledger_exact(gst), idx
            assert gst["histories"] == N_GPU
            # per voxel, where the oracle has events (its expected relative sigma,
            # from the independent run scaled to the oracle's history count)
            with np.errstate(divide="ignore", invalid="ignore"):
                rel_o = np.where(ds > 0, ss / ds, np.inf) * np.sqrt(N_GPU / N_ORACLE)
            dense = (ds > 0.1 * ds.max()) & (rel_o < 0.1)
            z = (dg - do)[dense] / np.sqrt(sg ** 2 + so ** 2)[dense]
            rates[idx] = (float(np.mean(np.abs(z) <= 3.0)) if z.size else 1.0, int(dense.sum()))
            zs.append(z)
            # per block of B^3 voxels: mass-weighted doses, Gy per history
            mb = _blocks(rho, n)
            with np.errstate(divide="ignore", invalid="ignore"):
                gb = _blocks(dg * rho, n) / mb
                sb = _blocks(ds * rho, n) / mb
                ob = oparts * (oracle.MEV_PER_G_TO_GY / (vol[idx] * mb))
            pick = sb > 0.1 * np.nanmax(sb)
            om, ose = ob.mean(0)[pick], ob.std(0, ddof=1)[pick] / np.sqrt(K)
            zb = (gb[pick] - om) / (ose * np.sqrt(1.0 + N_ORACLE / N_GPU))
            brates[idx] = (float(np.mean(np.abs(zb) <= 4.0)), int(pick.sum()))
            # a sequence's event counters go to its first plan: pool them by type
            t = specs[idx].particle
            for k_g, k_o in (("n_photon_real", "n_photon_real"), ("n_electron_steps", "n_e_steps_voxel_form"),
                             ("n_hard_real", "n_hard_real"), ("n_compton", "n_compton"),
                             ("n_pair", "n_pair"), ("n_brem", "n_brem"), ("n_moller", "n_moller")):
                c = counts[t].setdefault(k_g, [0, 0.0])
                c[0] += gst[k_g]
                c[1] += ost[k_o]
    finally:
        pool.terminate()
    ctx.close()
    assert len(rates) == len(specs) == len(brates)
    bad = {i: r for i, r in rates.items() if r[1] >= 30 and r[0] < 0.97}
    assert not bad, bad
    n_dense = sum(r[1] for r in rates.values())
    assert n_dense > 2_000, n_dense
    pooled = sum(r[0] * r[1] for r in rates.values()) / n_dense
    assert pooled >= 0.99, pooled
    bad = {i: r for i, r in brates.items() if r[1] >= 50 and r[0] < 0.97}
    assert not bad, bad
    assert sum(1 for r in brates.values() if r[1] >= 50) >= 48  # the block test reaches most plans
    bpooled = sum(r[0] * r[1] for r in brates.values()) / sum(r[1] for r in brates.values())
    assert bpooled >= 0.985, bpooled
    z = np.concatenate(zs)
    assert abs(float(np.mean(z))) < 0.1, (float(np.mean(z)), float(np.std(z)), z.size)
    assert 0.85 < float(np.std(z)) < 1.15, (float(np.mean(z)), float(np.std(z)), z.size)
    for t in (0, 1):
        n_plans = sum(1 for sp in specs if sp.particle == t)
        for k, (g_count, o_count) in counts[t].items():
            if o_count < 2000:
                continue
            g_rate = g_count / (N_GPU * n_plans)
            o_rate = o_count / (N_ORACLE * n_plans)
            assert g_rate == pytest.approx(o_rate, rel=0.03), (t, k, g_rate, o_rate)


@pytest.mark.parametrize("index,n,n_ora", [(28, 84, 8_000_000), (14, 64, 3_000_000)])
def test_batched_workload_electron_plan_gamma(index, n, n_ora):
    """Gamma 2% / 2 mm (voxels above 20% of D_max, the oracle as reference) on
    electron plans of the batched workload: plan 28, 84^3 voxels of 0.467 cm
    with a 12.5 MeV field of 10.7 cm, and plan 14, 64^3 voxels of 0.377 cm with
    a 7.1 MeV field of 3.9 cm, both on smoothed-noise densities of 0.2 to 2.0
    g/cm^3.  The oracle's histories bring its noise in the high-dose region
    under 1% of D_max; the GPU runs five times more.  (A photon plan would need
    over 1e8 oracle histories for that: its low-density voxels see few
    interactions.)"""
    import torch

    sp = W.config4()[index]
    assert sp.particle == W.ELECTRON and sp.n == n
    ph = sp.phantom()
    src = W.square_field(sp.particle, sp.energy, ph, sp.field_cm)
    ctx = make_ctx()
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, src, sp.seed, 16)
    ctx.run([plan], [5 * n_ora])
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(d)
    st = ctx.plan_result(plan, 0.5, d.data_ptr(), s.data_ptr())
    assert ledger_exact(st)
    dg, sg = d.cpu().numpy(), s.cpu().numpy()
    ctx.close()
    ora = oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, n_ora, 123, processes=host_cores())
    do, so = ora.dose_gy(ph), ora.sigma_gy(ph)
    noise = float(np.median(so[do > 0.5 * do.max()] / do.max()))
    rate = gamma_pass_rate(do.reshape(n, n, n), dg.reshape(n, n, n), (10.0 * sp.voxel_cm,) * 3)
    assert noise < 0.01, (noise, rate)
    assert three_sigma_pass_rate(dg, sg, do, so, dg > 0.1 * dg.max()) >= 0.99
    assert rate >= 0.98, (rate, noise)

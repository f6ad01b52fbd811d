#!/usr/bin/env python
"""Benchmark: histories/s of the coupled photon-electron transport on the
paper's timing workload (GPUMCD §II.D / Table "resabsexec"): separate 15 MeV
10x10 cm^2 parallel beams of 1e6 electrons and 4e6 photons on a 128^3 water
phantom at 0.25 cm.  One step = both beams, each run from a zeroed tally to
its FP64 dose and uncertainty on the device.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
histories (weak scaling, no data-path collective); the time is the max over
ranks.  ``--impl reference`` times the FP64 CPU oracle on the host cores
instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "histories/s (1e6 e- + 4e6 photons, 15 MeV, 128^3 water, to FP64 dose + sigma)"
UNIT = "histories/s"
N_E, N_G = 1_000_000, 4_000_000



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run each beam once at 1/5 of its histories (small case for ncu) and exit")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "batched", "served", "geoms", "ablation", "kerma", "grouping"],
                    help="c2: the contract line; batched: 64 uneven plans in one launch vs alone; "
                         "served: a Poisson request stream with continuous batching; geoms: the "
                         "paper's three geometries, each beam alone (Table resabsexec); ablation: "
                         "the lane refill policies on the second geometry (Table resdivred); "
                         "kerma: the photon-only mode against full transport on the c2 photon beam; "
                         "grouping: polyenergetic phase spaces and spectra, ungrouped vs grouped by energy")
    ap.add_argument("--small", action="store_true",
                    help="ablation, grouping: 1/5 of the histories (a small case for ncu)")
    ap.add_argument("--graph", action="store_true",
                    help="launch each sequence's first launch from a captured CUDA graph")
    ap.add_argument("--requests", type=int, default=1000, help="served: number of requests")
    ap.add_argument("--round-histories", type=int, default=16_000_000,
                    help="served: histories per round over all active plans")
    ap.add_argument("--rounds-in-flight", type=int, default=2, help="served: rounds on the device at once")
    ap.add_argument("--calibration", type=int, default=48,
                    help="served: requests of the capacity run (served vs alone)")
    ap.add_argument("--target", type=float, default=0.01, help="served: relative uncertainty target")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served: HBM budget")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(
        os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_sample(seconds: float = 12.0, seed0: int = 100):
    """Times the FP64 oracle (as it stands) on bounded samples of the workload
    over all host cores: electrons and photons in the 1:4 ratio of the step.
    Returns (histories/s, cores, description)."""
    import oracle
    import workloads as W

    cores = host_cores()
    pe, pg = W.config2(W.ELECTRON), W.config2(W.PHOTON)
    n_e, n_g = 150 * cores, 600 * cores
    done = 0
    t0 = time.perf_counter()
    rounds = 0
    while True:
        oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, pe.phantom, pe.source, n_e, seed0 + rounds,
                        processes=cores)
        oracle.simulate(W.MATERIALS, W.DEFAULT_PHYSICS, pg.phantom, pg.source, n_g, seed0 + rounds,
                        processes=cores)
        done += n_e + n_g
        rounds += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    desc = (f"{rounds} round(s) of {n_e} e- + {n_g} photons (15 MeV, 10x10 cm^2, 128^3 water), "
            f"{cores} processes")
    return done / dt, cores, desc


def rank_seed(rank: int, step: int) -> int:
    """Seed of a rank's step: every rank simulates its own, disjoint histories."""
    return 1_000_003 * (rank + 1) + 2 * step


def max_over_ranks(value: float, dist, device) -> float:
    """The timed region's length is the slowest rank's (barrier-bracketed)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(seconds=3.0)
    vals, descs, cores = [], None, host_cores()
    t_all = 0.0
    for i in range(args.steps):
        v, cores, descs = oracle_sample(seconds=8.0, seed0=1000 + 10 * i)
        vals.append(v)
        t_all += (N_E + N_G) / v
    value = (N_E + N_G) * args.steps / t_all
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": "c2_water128_15MeV_e1e6_photon4e6", "parallelism": "host cores"},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": descs},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_ours(args):
    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()  # spawned processes, before the GPU work starts

    pe, pg = W.config2(W.ELECTRON), W.config2(W.PHOTON)
    nvox = pe.phantom.nvox
    ctx = g.engine(local)
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    pid = ctx.create_phantom(pe.phantom)
    plan_e = ctx.plan_open(pid, pe.source, 1, 32)
    plan_g = ctx.plan_open(pid, pg.source, 2, 32)
    out = {k: torch.empty(nvox, dtype=torch.float64, device=dev) for k in ("de", "se", "dg", "sg")}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 2x the 129 MB L2

    def step(i):
        se = rank_seed(rank, i)
        ctx.plan_reset(plan_e, se, sh)
        ctx.run([plan_e], [N_E], sh)
        st_e = ctx.plan_result(plan_e, 0.5, out["de"].data_ptr(), out["se"].data_ptr(), sh)
        ctx.plan_reset(plan_g, se + 1, sh)
        ctx.run([plan_g], [N_G], sh)
        st_g = ctx.plan_result(plan_g, 0.5, out["dg"].data_ptr(), out["sg"].data_ptr(), sh)
        return st_e, st_g

    for i in range(args.warmup):
        step(-1 - i)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush between timed steps (outside the events)
                ev[i][0].record(stream)
                stats.append(step(i))
                ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = (N_E + N_G) * args.steps * world / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: each step uploads the
    # phantom from pinned host memory, runs both beams through gpumcd_simulate
    # and reads dose and sigma back into pinned host memory
    import numpy as np

    import workloads as W

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    ph_host = W.Phantom(pe.phantom.dims, pe.phantom.voxel_cm, pinned(pe.phantom.mat), pinned(pe.phantom.rho))
    hd = {k: torch.empty(nvox, dtype=torch.float64, pin_memory=True).numpy() for k in ("de", "se", "dg", "sg")}

    def e2e_step(i):
        p2 = ctx.create_phantom(ph_host)
        ctx.simulate(p2, pe.source, N_E, 77 + i, nvox=nvox, out=(hd["de"], hd["se"]))
        ctx.simulate(p2, pg.source, N_G, 78 + i, nvox=nvox, out=(hd["dg"], hd["sg"]))
        ctx.destroy_phantom(p2)

    e2e_step(-1)  # warm-up, like the device metric's
    e2e_t = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step(i)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = (N_E + N_G) * world / statistics.median(e2e_t)
    h2d = pe.phantom.mat.nbytes + pe.phantom.rho.nbytes
    d2h = 4 * nvox * 8

    st_e, st_g = stats[-1]
    launches = st_e["n_launches"] + st_g["n_launches"] + 2 * 3  # transport + fold, s_thr, ledger sum
    clocks = clk.summary()
    ev_e = st_e["n_electron_steps"] + st_e["n_photon_events"]
    ev_g = st_g["n_electron_steps"] + st_g["n_photon_events"]
    kern_ms = st_e["transport_ms"] + st_g["transport_ms"]
    import paper_1101_1245_gb300.roofline as rl
    roof = rl.alu_roofline(ev_e, ev_g, kern_ms, clocks.get("sm_mhz"),
                           torch.cuda.get_device_properties(dev).multi_processor_count,
                           launches=st_e["n_launches"] + st_g["n_launches"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2_water128_15MeV_e1e6_photon4e6",
                       "phantom": "128^3 water, 0.25 cm", "beams": "15 MeV 10x10 cm^2 e- 1e6, photons 4e6",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "launch_graph": bool(args.graph),
                       "s05_electron": st_e["s_thr"], "s05_photon": st_g["s_thr"],
                       "transport_ms_electron": st_e["transport_ms"],
                       "transport_ms_photon": st_g["transport_ms"],
                       "ledger_exact": all(s["e_deposited"] + s["e_escaped"] + s["e_rest"] == s["e_incident"]
                                           for s in (st_e, st_g))},
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "host_memory": "pinned"},
            "gpu_launches": launches,
            "clocks": clocks}
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": UNIT, "cores": cpu[1], "kind": "oracle",
                                "sample": cpu[2]}
    if rank == 0:
        emit(line)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def _c4_phantom(spec):
    ph = spec.phantom()
    return ph.dims, ph.voxel_cm, ph.mat, ph.rho


def c4_phantoms(specs):
    """The seeded C4 phantoms, generated over the host cores (spawned workers)."""
    import multiprocessing as mp

    import workloads as W
    with mp.get_context("spawn").Pool(min(host_cores(), len(specs))) as pool:
        parts = pool.map(_c4_phantom, specs)
    return [W.Phantom(d, v, m, r) for d, v, m, r in parts]


def run_batched(args):
    """Config 4: 64 independent uneven plans in one batched persistent launch
    (autotuned), against the same plans run one by one."""
    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W
    from paper_1101_1245_gb300.autotune import autotune

    specs = W.config4()
    phantoms = c4_phantoms(specs)
    ctx = g.engine(0)
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    pids = [ctx.create_phantom(ph) for ph in phantoms]
    srcs = [W.square_field(sp.particle, sp.energy, ph, sp.field_cm) for sp, ph in zip(specs, phantoms)]
    nh = [-(-sp.n_histories // 16) * 16 for sp in specs]  # whole multiples of the 16 batches
    # the tuner times the whole plan set at 1/8 of its histories in one launch,
    # so a trial is tens of ms and the launch tail weighs as it does at full size
    sample = [(pids[i], srcs[i], max(16, nh[i] // 8 // 16 * 16)) for i in range(len(specs))]
    default_launch = ctx.get_launch()
    tuned = autotune(ctx, sample, reps=2)
    plans = [ctx.plan_open(pid, src, sp.seed, 16) for pid, src, sp in zip(pids, srcs, specs)]
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def batched():
        for p, sp in zip(plans, specs):
            ctx.plan_reset(p, sp.seed)
        torch.cuda.synchronize()
        ev[0].record()
        ctx.run(plans, nh)
        st = [ctx.plan_result(p, 0.5) for p in plans]
        ev[1].record()
        torch.cuda.synchronize()
        # a set of both particle types runs as one sequence per type: its
        # transport time is the sum of the two sequences'
        per_type = {sp.particle: x["transport_ms"] for sp, x in zip(specs, st)}
        return ev[0].elapsed_time(ev[1]), sum(per_type.values()), st

    def plain():
        tot = tr = 0.0
        for p, sp, n in zip(plans, specs, nh):
            ctx.plan_reset(p, sp.seed)
            torch.cuda.synchronize()
            ev[0].record()
            ctx.run([p], [n])
            tr += ctx.plan_result(p, 0.5)["transport_ms"]
            ev[1].record()
            torch.cuda.synchronize()
            tot += ev[0].elapsed_time(ev[1])
        return tot, tr

    for _ in range(max(1, args.warmup)):
        batched()
        plain()
    rb = [batched()[:2] for _ in range(args.steps)]
    rp = [plain() for _ in range(args.steps)]
    tb, tbt = statistics.median(r[0] for r in rb), statistics.median(r[1] for r in rb)
    tp_tuned, tpt_tuned = statistics.median(r[0] for r in rp), statistics.median(r[1] for r in rp)
    st = batched()[2]
    # the plain form also at the default launch: the tuner picks for the
    # batched launch, and a setting that suits it (larger chunks) can slow the
    # single-plan runs; the plain side is credited with the better of the two
    tuned_launch = ctx.get_launch()
    ctx.set_launch(**default_launch)
    plain()
    rp_def = [plain() for _ in range(args.steps)]
    ctx.set_launch(**tuned_launch)
    tp_def, tpt_def = statistics.median(r[0] for r in rp_def), statistics.median(r[1] for r in rp_def)
    tp, tpt = min(tp_tuned, tp_def), min(tpt_tuned, tpt_def)
    total = sum(nh)
    emit({"workload": "c4_batched_64_plans", "metric": "histories/s (64 uneven plans, to FP64 dose + sigma)",
          "unit": UNIT, "batched_value": total / (tb / 1e3), "plain_value": total / (tp / 1e3),
          "batched_over_plain": tp / tb, "batched_ms": tb, "plain_ms": tp,
          "batched_transport_ms": tbt, "plain_transport_ms": tpt,
          "batched_over_plain_transport": tpt / tbt, "histories": total,
          "plain_basis": "the better of the tuned and the default launch, per measure",
          "plain_ms_tuned_launch": tp_tuned, "plain_ms_default_launch": tp_def,
          "plain_transport_ms_tuned_launch": tpt_tuned, "plain_transport_ms_default_launch": tpt_def,
          "plans": len(plans), "voxels": int(sum(ph.nvox for ph in phantoms)),
          "electron_plans": int(sum(sp.particle for sp in specs)),
          "ledger_exact": all(x["e_deposited"] + x["e_escaped"] + x["e_rest"] == x["e_incident"] for x in st),
          "autotuned_launch": tuned["launch"], "autotune_trials": len(tuned["trials"]),
          "n_batches": 16, "steps": args.steps, "launch_graph": bool(args.graph), "data": "synthetic"})
    ctx.close()


# GPUMCD Table "resabsexec" (GTX480, seconds for 1e6 electrons / 4e6 photons at
# 15 MeV), quoted beside the GB300 times as context only
PAPER_ABSEXEC_S = {("geom1", "electron"): 0.118, ("geom2", "electron"): 0.147, ("geom3", "electron"): 0.162,
                   ("geom1", "photon"): 0.269, ("geom2", "photon"): 0.275, ("geom3", "photon"): 0.366}


def run_geoms(args):
    """The paper's three geometries (GPUMCD §III.A) with its timing beams: the
    water phantom (the c2 workload), the lung box and the tissue / lung / bone
    slabs, each beam run alone from a zeroed tally to FP64 dose and sigma.
    Also reports the share of fictitious events, which the bone slab's
    majorant drives up."""
    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0, mats=W.MATERIALS_PAPER)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    rows = []
    for geom, make in (("geom1", W.config2), ("geom2", W.geom2), ("geom3", W.geom3),
                       ("synthetic_ct", W.synthetic_ct)):
        for particle in (W.ELECTRON, W.PHOTON):
            pl = make(particle)
            pid = ctx.create_phantom(pl.phantom)
            plan = ctx.plan_open(pid, pl.source, pl.seed, 32)

            def once(seed):
                ctx.plan_reset(plan, seed)
                torch.cuda.synchronize()
                ev[0].record()
                ctx.run([plan], [pl.n_histories])
                st = ctx.plan_result(plan, 0.5)
                ev[1].record()
                torch.cuda.synchronize()
                return ev[0].elapsed_time(ev[1]), st

            for i in range(max(1, args.warmup)):
                once(1000 + i)
            res = [once(2000 + i) for i in range(args.steps)]
            ms = statistics.median(r[0] for r in res)
            st = res[-1][1]
            name = "electron" if particle == W.ELECTRON else "photon"
            ph_ev = st["n_photon_events"]
            hard = st["n_hard_real"] + st["n_hard_fict"]
            rows.append({"geometry": geom, "beam": name, "histories": pl.n_histories, "ms": ms,
                         "transport_ms": statistics.median(r[1]["transport_ms"] for r in res),
                         "histories_per_s": pl.n_histories / (ms / 1e3),
                         "paper_gtx480_s": PAPER_ABSEXEC_S.get((geom, name)),
                         "photon_fictitious_share": (ph_ev - st["n_photon_real"]) / ph_ev if ph_ev else 0.0,
                         "hard_fictitious_share": st["n_hard_fict"] / hard if hard else 0.0,
                         "electron_steps_per_history": st["n_electron_steps"] / pl.n_histories,
                         "ledger_exact": st["e_deposited"] + st["e_escaped"] + st["e_rest"] == st["e_incident"]})
            ctx.plan_close(plan)
            ctx.destroy_phantom(pid)
    ctx.close()
    emit({"workload": "paper_geometries_15MeV", "metric": "ms per beam (1e6 e- or 4e6 photons, to FP64 dose + sigma)",
          "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
          "phantoms": "128^3 at 0.25 cm: water; lung box in water; tissue/lung/bone slabs; "
                      "synthetic-CT thorax 128x96x128 (6 MV-like photons, 15 MeV electrons)",
          "data": "synthetic", "rows": rows})


# GPUMCD Table "resdivred" (GTX480, geometry 2): base time in seconds and the
# accelerations of stream compaction and of the persistent pool, as context
PAPER_DIVRED = {"electron": {"t_base_s": 0.185, "a_comp": 1.06, "a_pool": 1.26},
                "photon": {"t_base_s": 0.275, "a_comp": 0.85, "a_pool": 0.98}}


def run_ablation(args):
    """Divergence-reduction ablation (GPUMCD §II.C.3, Table resdivred) on the
    paper's second geometry with its timing beams: the lane refill policies of
    the persistent kernel.  base = a warp's lanes refill only when all are
    empty; comp N = every N-th pass (the paper's compaction after N steps);
    pool = every pass (the production policy).  Tallies are identical under
    every policy, which the line checks."""
    import hashlib

    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0)
    policies = [("base", g.REFILL_WHEN_EMPTY), ("comp64", 64), ("comp16", 16), ("comp4", 4), ("pool", 1)]
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    rows = []
    for particle in (W.ELECTRON, W.PHOTON):
        pl = W.geom2(particle)
        if args.small:
            pl.n_histories //= 5
        pid = ctx.create_phantom(pl.phantom)
        plan = ctx.plan_open(pid, pl.source, pl.seed, 32)
        d = torch.zeros(pl.phantom.nvox, dtype=torch.float64, device="cuda")
        sg = torch.zeros_like(d)
        name = "electron" if particle == W.ELECTRON else "photon"
        times, hashes = {}, set()
        for label, period in policies:
            ctx.set_launch(refill_period=period)

            def once(seed):
                ctx.plan_reset(plan, seed)
                torch.cuda.synchronize()
                ev[0].record()
                ctx.run([plan], [pl.n_histories])
                st = ctx.plan_result(plan, 0.5, d.data_ptr(), sg.data_ptr())
                ev[1].record()
                torch.cuda.synchronize()
                return ev[0].elapsed_time(ev[1]), st["transport_ms"]

            for i in range(max(1, args.warmup)):
                once(pl.seed)
            res = [once(pl.seed) for _ in range(args.steps)]
            hashes.add(hashlib.sha256(d.cpu().numpy().tobytes() + sg.cpu().numpy().tobytes()).hexdigest())
            times[label] = (statistics.median(r[0] for r in res), statistics.median(r[1] for r in res))
        ctx.set_launch(refill_period=1)
        tb = times["base"][1]
        rows.append({"beam": name, "histories": pl.n_histories,
                     "transport_ms": {k: v[1] for k, v in times.items()},
                     "step_ms": {k: v[0] for k, v in times.items()},
                     "a_comp": {k: tb / times[k][1] for k in ("comp64", "comp16", "comp4")},
                     "a_pool": tb / times["pool"][1],
                     "tallies_identical": len(hashes) == 1,
                     "paper_gtx480": PAPER_DIVRED[name]})
        ctx.plan_close(plan)
        ctx.destroy_phantom(pid)
    ctx.close()
    emit({"workload": "ablation_refill_policy_geom2_15MeV",
          "metric": "transport ms per beam under each lane refill policy; A = T_base / T",
          "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
          "phantom": "lung box in water, 128^3 at 0.25 cm", "data": "synthetic", "rows": rows})


def run_kerma(args):
    """The photon-only mode (GPUMCD_LAUNCH_KERMA) against full coupled
    transport on the c2 photon beam (15 MeV, 4e6 photons, 128^3 water): time,
    and the central-axis depth dose of each (mean over the central 1x1 cm)."""
    import numpy as np
    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0)
    pl = W.config2(W.PHOTON)
    ph = pl.phantom
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, pl.source, pl.seed, 32)
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    sg = torch.zeros_like(d)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    nx, ny, nz = ph.dims
    h = 2  # central 1x1 cm at 0.25 cm voxels
    out = {}
    for label, flags in (("transport", 0), ("kerma", g.LAUNCH_KERMA)):
        ctx.set_launch(flags=flags)

        def once():
            ctx.plan_reset(plan, pl.seed)
            torch.cuda.synchronize()
            ev[0].record()
            ctx.run([plan], [pl.n_histories])
            st = ctx.plan_result(plan, 0.5, d.data_ptr(), sg.data_ptr())
            ev[1].record()
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]), st

        for _ in range(max(1, args.warmup)):
            once()
        res = [once() for _ in range(args.steps)]
        dose = d.cpu().numpy().reshape(nz, ny, nx)
        pdd = dose[:, ny // 2 - h:ny // 2 + h, nx // 2 - h:nx // 2 + h].mean(axis=(1, 2))
        st = res[-1][1]
        out[label] = {"ms": statistics.median(r[0] for r in res),
                      "transport_ms": statistics.median(r[1]["transport_ms"] for r in res),
                      "electron_steps": st["n_electron_steps"], "pdd": pdd}
    ctx.set_launch(flags=0)
    ctx.close()
    t, k = out["transport"], out["kerma"]
    depths = [0.125, 1.125, 3.125, 5.125, 10.125, 20.125]  # voxel centres, cm
    norm = t["pdd"].max()
    emit({"workload": "c2_photon_kerma_vs_transport", "metric": "ms per beam and central-axis dose",
          "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
          "histories": pl.n_histories, "data": "synthetic",
          "transport_ms": t["transport_ms"], "kerma_ms": k["transport_ms"],
          "speedup": t["transport_ms"] / k["transport_ms"],
          "step_ms": {"transport": t["ms"], "kerma": k["ms"]},
          "electron_steps": {"transport": t["electron_steps"], "kerma": k["electron_steps"]},
          "depth_of_max_cm": {"transport": float(np.argmax(t["pdd"]) * 0.25 + 0.125),
                              "kerma": float(np.argmax(k["pdd"]) * 0.25 + 0.125)},
          "pdd_over_transport_max": {f"{z:g}": {"transport": float(t["pdd"][int(z / 0.25)] / norm),
                                                "kerma": float(k["pdd"][int(z / 0.25)] / norm)}
                                     for z in depths}})


def run_grouping(args):
    """Energy grouping of polyenergetic beams (GPUMCD §IV) on the c2 phantom
    (128^3 water), with the paper's timing history counts, each source
    ungrouped against grouped (energy_grouping):
    - a phase space of 1e6 records in random order (6 MV-like photons, 1-15
      MeV electrons), used as listed or stably sorted by decreasing energy;
    - a 10x10 cm^2 field whose spectrum (the same energies) is sampled on the
      device, iid or stratified over the run from the top down.
    The two forms give different, equally valid samples of the same dose; the
    line reports the share of voxels above 10% of the maximum where they agree
    within 3 combined sigma."""
    import numpy as np
    import torch

    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    rows = []
    for kind in ("phase_space", "spectrum"):
        for particle in (W.ELECTRON, W.PHOTON):
            pl = W.config2(particle)
            if args.small:
                pl.n_histories //= 5
            ph = pl.phantom
            pid = ctx.create_phantom(ph)
            if kind == "phase_space":
                src = W.polyenergetic_phase_space(particle, ph, 1_000_000, seed=77)
            else:
                src = W.polyenergetic_square(particle, ph)
            d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
            sg = torch.zeros_like(d)
            out = {}
            for label, grouping in (("ungrouped", W.ENERGY_UNGROUPED), ("grouped", W.ENERGY_GROUPED)):
                src.energy_grouping = grouping
                plan = ctx.plan_open(pid, src, pl.seed, 32)

                def once():
                    ctx.plan_reset(plan, pl.seed)
                    torch.cuda.synchronize()
                    ev[0].record()
                    ctx.run([plan], [pl.n_histories])
                    st = ctx.plan_result(plan, 0.5, d.data_ptr(), sg.data_ptr())
                    ev[1].record()
                    torch.cuda.synchronize()
                    return ev[0].elapsed_time(ev[1]), st

                for _ in range(max(1, args.warmup)):
                    once()
                res = [once() for _ in range(args.steps)]
                st = res[-1][1]
                out[label] = {"ms": statistics.median(r[0] for r in res),
                              "transport_ms": statistics.median(r[1]["transport_ms"] for r in res),
                              "electron_steps_per_history": st["n_electron_steps"] / pl.n_histories,
                              "ledger_exact": st["e_deposited"] + st["e_escaped"] + st["e_rest"] == st["e_incident"],
                              "dose": d.cpu().numpy(), "sigma": sg.cpu().numpy()}
                ctx.plan_close(plan)
            ctx.destroy_phantom(pid)
            a, b = out["ungrouped"], out["grouped"]
            mask = a["dose"] > 0.1 * a["dose"].max()
            agree = np.abs(a["dose"] - b["dose"]) <= 3.0 * np.sqrt(a["sigma"] ** 2 + b["sigma"] ** 2)
            rows.append({"source": kind, "beam": "electron" if particle == W.ELECTRON else "photon",
                         "histories": pl.n_histories,
                         "transport_ms": {k: v["transport_ms"] for k, v in out.items()},
                         "step_ms": {k: v["ms"] for k, v in out.items()},
                         "grouped_speedup": a["transport_ms"] / b["transport_ms"],
                         "electron_steps_per_history": {k: v["electron_steps_per_history"] for k, v in out.items()},
                         "ledger_exact": all(v["ledger_exact"] for v in out.values()),
                         "dose_3sigma_agreement": float(agree[mask].mean())})
    ctx.close()
    emit({"workload": "polyenergetic_energy_grouping_c2_phantom",
          "metric": "transport ms per beam, ungrouped vs grouped by energy",
          "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
          "phantom": "128^3 water at 0.25 cm", "data": "synthetic", "rows": rows})


def run_served(args):
    """Config 5: a Poisson stream of dose requests from the config-4
    distribution on resident phantoms, served with continuous batching to a
    relative uncertainty target over voxels above 50% of D_max; against the
    same requests run one by one."""
    import numpy as np

    import paper_1101_1245_gb300 as g
    import workloads as W
    from paper_1101_1245_gb300.serve import DoseRequest, Server, run_alone

    pool_specs = W.config4()
    phantoms = c4_phantoms(pool_specs)
    budget = int(args.budget_gb * 2 ** 30)
    ctx = g.engine(0, hbm_budget_bytes=budget + (8 << 30))
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    pids = [ctx.create_phantom(ph) for ph in phantoms]

    def requests(rate):
        reqs = []
        for i, r in enumerate(W.config5(count=args.requests, rate_per_s=rate)):
            k = i % len(phantoms)
            ph, sp = phantoms[k], r.spec
            src = W.square_field(sp.particle, sp.energy, ph, sp.field_cm)
            reqs.append(DoseRequest(i, pids[k], ph.nvox, src, sp.seed, r.arrival_s, 400_000_000))
        return reqs

    # capacity: a calibration set all present at once, served, against the
    # same requests run one at a time with the plain kernel
    cal = requests(1.0)[:min(args.calibration, args.requests)]
    srv = Server(ctx, budget, target=args.target, round_histories=args.round_histories,
                 rounds_in_flight=args.rounds_in_flight)
    for q in cal:
        srv.submit(q)
    srv.run(real_time=False)
    rep_cal = srv.report()
    alone = [run_alone(ctx, q, args.target) for q in cal]
    alone_h = sum(a.histories for a in alone)
    alone_t = sum(a.done_s for a in alone)
    mean_h = rep_cal["histories"] / max(rep_cal["requests"], 1)
    rate = 0.8 * rep_cal["histories_per_s"] / mean_h
    # the stream: Poisson arrivals at 0.8 x that capacity
    srv = Server(ctx, budget, target=args.target, round_histories=args.round_histories,
                 rounds_in_flight=args.rounds_in_flight)
    reqs = requests(rate)
    for q in reqs:
        srv.submit(q)
    srv.run(real_time=True)
    rep = srv.report()
    emit({"workload": "c5_served", "metric": "histories/s and request latency at s_0.5 <= target",
          "unit": UNIT, "target": args.target, "threshold": 0.5,
          "served_capacity_value": rep_cal["histories_per_s"],
          "alone_value": alone_h / alone_t if alone_t else None,
          "served_over_alone": rep_cal["histories_per_s"] * alone_t / alone_h if alone_h else None,
          "capacity_requests": len(cal), "capacity_histories": rep_cal["histories"],
          "alone_histories": alone_h, "capacity_rounds": rep_cal["rounds"],
          "requests": rep["requests"], "arrival_rate_per_s": rate,
          "rate_basis": "0.8 x the served capacity on the calibration set",
          "stream_value": rep["histories_per_s"], "latency_p50_s": rep["latency_p50_s"],
          "latency_p99_s": rep["latency_p99_s"], "wall_s": rep["wall_s"], "rounds": rep["rounds"],
          "folds": rep["folds"], "mean_histories_per_request": rep["histories"] / max(rep["requests"], 1),
          "s_thr_max": rep["s_thr_max"], "rounds_in_flight": args.rounds_in_flight,
          "round_histories": args.round_histories, "hbm_budget_gb": args.budget_gb,
          "launch_graph": bool(args.graph),
          "phantoms": "64 resident config-4 phantoms, request i on phantom i mod 64", "data": "synthetic"})
    ctx.close()


def run_ncu_case():
    """Each beam of the step once at 1/5 of its histories, untimed: the small
    case profiled with ncu --set full (one launch of the transport kernel per beam)."""
    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0)
    for part, n in ((W.ELECTRON, N_E // 5), (W.PHOTON, N_G // 5)):
        pl = W.config2(part)
        pid = ctx.create_phantom(pl.phantom)
        plan = ctx.plan_open(pid, pl.source, 5, 32)
        ctx.run([plan], [n])
        st = ctx.plan_result(plan, 0.5)
        print(json.dumps({"case": pl.name, "histories": n, **{k: st[k] for k in (
            "n_electron_steps", "n_photon_events", "n_hard_real", "n_launches", "transport_ms")}}),
            flush=True)
        ctx.plan_close(plan)
        ctx.destroy_phantom(pid)
    ctx.close()


def main():
    args = parse()
    if args.ncu_case:
        run_ncu_case()
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "geoms":
        run_geoms(args)
        return
    if args.workload == "ablation":
        run_ablation(args)
        return
    if args.workload == "kerma":
        run_kerma(args)
        return
    if args.workload == "grouping":
        run_grouping(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark: histories/s at 1% dose uncertainty, plain vs batched vs served,
with p50/p99 request latency (GPUMCD §II.D: the uncertainty s over voxels
above half of D_max).

Default workload: the batched configuration, 64 independent uneven plans
(64^3 to 256^3 voxels of 0.2 to 0.5 cm, smoothed-noise densities of 0.2 to
2.0 g/cm^3, 6 to 18 MeV photon or electron fields of 2 to 15 cm), each run
from a zeroed tally to s_0.5 <= 1% (gpumcd_run_to_uncertainty: a first round
of the plan's own history count, then rounds sized by s ~ 1/sqrt(N)).  One
step = all 64 plans to 1%.
- value: the batched form: in each round a plan given >= 2^23 histories runs in a
  launch of its own, the other active plans share one launch
  sequence per particle type;
- plain: the same plans one at a time with the same schedule (the same
  histories and, bit for bit, the same tallies);
- served: a Poisson stream of 1000 requests from the same distribution on
  resident phantoms with continuous batching (serve.py), p50/p99 latency;
- the paper's timing workload (1e6 e- + 4e6 photons, 15 MeV, 128^3 water) and
  the heterogeneous slab configuration (1e7 photons of a 6 MV-like spectrum on
  256^3, ungrouped and grouped by energy, also run to 1%) as sub-records.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c4|c2|batched|served|geoms|ablation|kerma|grouping]

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

METRIC = "histories/s at 1% dose uncertainty (plain vs batched/served); p50/p99 latency"
METRIC_C2 = "histories/s (1e6 e- + 4e6 photons, 15 MeV, 128^3 water, to FP64 dose + sigma)"
UNIT = "histories/s"
N_E, N_G = 1_000_000, 4_000_000
TARGET, THRESHOLD = 0.01, 0.5   # s_0.5 <= 1%
W_C4 = 16                       # batch tallies per plan of the batched workload
# ...and of the timing workload's beams: half the tally of 32 batches (268 MB
# for 128^3), 3% faster transport (fewer L2 misses on the tally), with 15
# degrees of freedom for sigma
W_C2 = 16
CAP_C4 = 400_000_000            # histories per plan at most
# the slab configuration's s_0.5 is ~12% at its 1e7 histories (0.2 cm voxels):
# 1% takes ~1.5e9
CAP_C3 = 2_000_000_000

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run each beam once at 1/5 of its histories (small case for ncu) and exit")
    ap.add_argument("--workload", default="c4",
                    choices=["c4", "c2", "batched", "served", "geoms", "ablation", "kerma", "grouping"],
                    help="c4: the contract line (64 uneven plans to 1%%, batched vs plain vs served); "
                         "c2: the paper's timing workload alone; "
                         "batched: 64 uneven plans in one launch vs alone at fixed histories; "
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
    ap.add_argument("--no-served", action="store_true", help="c4: leave out the served stream")
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


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_job(job):
    """Worker: the oracle, as it stands, on one sample (a workload's phantom and
    beam, n histories).  An empty run of the same set-up is timed too and
    subtracted, so the figure is the cost per history of a long run."""
    import oracle
    import workloads as W

    kind, key, n, seed = job
    if kind == "c4":
        spec = W.config4()[key]
        ph = spec.phantom()
        src = W.square_field(spec.particle, spec.energy, ph, spec.field_cm)
    else:
        pl = W.config2(key)
        ph, src = pl.phantom, pl.source
    t0 = time.perf_counter()
    oracle.simulate_range(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, 0, 0, seed)
    t1 = time.perf_counter()
    oracle.simulate_range(W.MATERIALS, W.DEFAULT_PHYSICS, ph, src, 0, n, seed)
    t2 = time.perf_counter()
    return kind, key, n, max((t2 - t1) - (t1 - t0), 1e-9)


def oracle_rate(jobs, weights, cores: int):
    """Runs the sample jobs over `cores` spawned processes at once.  Returns
    (concurrent histories/s, one process's histories/s, histories timed, wall
    s): the per-history cost of each job's workload is weighted by the
    histories that workload holds in a step (weights[(kind, key)])."""
    import multiprocessing as mp

    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    cost = {}
    for kind, key, n, dt in out:
        c = cost.setdefault((kind, key), [0, 0.0])
        c[0] += n
        c[1] += dt
    tot_w = sum(weights[k] for k in cost)
    per_hist = sum(weights[k] * c[1] / c[0] for k, c in cost.items()) / tot_w
    one = 1.0 / per_hist
    return one * cores, one, sum(c[0] for c in cost.values()), wall


def c4_weights():
    """Histories of each plan's first round in the batched workload (the
    weights of the oracle's per-history costs)."""
    import workloads as W
    return {("c4", sp.index): -(-sp.n_histories // W_C4) * W_C4 for sp in W.config4()}


def oracle_sample_c4(per_plan: int = 1500, seed0: int = 100):
    """The FP64 oracle, as it stands, on a bounded sample of the batched
    workload: every plan at `per_plan` histories, one process per plan, all
    host cores at once; costs weighted by the plans' first-round histories."""
    import workloads as W
    cores = host_cores()
    jobs = [("c4", sp.index, per_plan, seed0 + sp.index) for sp in W.config4()]
    rate, one, n, wall = oracle_rate(jobs, c4_weights(), cores)
    desc = (f"{per_plan} histories of each of the 64 plans ({n} in all, {wall:.1f} s wall), one process "
            f"per plan over {cores} host cores, set-up excluded; per-history costs weighted by the plans' "
            f"first-round histories")
    return rate, one, cores, desc


def oracle_sample_c2(seed0: int = 100):
    """The oracle on a bounded sample of the paper's timing workload: 3000
    electrons and 12000 photons per host core, in the 1:4 ratio of the step."""
    import workloads as W
    cores = host_cores()
    jobs = []
    for i in range(cores):
        jobs.append(("c2", W.ELECTRON, 3000, seed0 + 2 * i))
        jobs.append(("c2", W.PHOTON, 12000, seed0 + 2 * i + 1))
    rate, one, n, wall = oracle_rate(jobs, {("c2", W.ELECTRON): N_E, ("c2", W.PHOTON): N_G}, cores)
    desc = (f"{cores} x (3000 e- + 12000 photons), 15 MeV, 10x10 cm^2, 128^3 water ({n} histories, {wall:.1f} s "
            f"wall) over {cores} host cores, set-up excluded")
    return rate, one, cores, desc


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
    """The oracle as it stands, timed on the host cores on bounded samples of
    the workload (each step one sample); rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    c2 = args.workload == "c2"
    sample = oracle_sample_c2 if c2 else oracle_sample_c4
    for i in range(args.warmup):
        sample(seed0=10 * (i + 1)) if c2 else sample(per_plan=300, seed0=10 * (i + 1))
    vals, ones, walls, desc, cores = [], [], [], None, host_cores()
    for i in range(args.steps):
        t0 = time.perf_counter()
        v, one, cores, desc = sample(seed0=1000 + 100 * i) if c2 else sample(per_plan=600, seed0=1000 + 100 * i)
        walls.append(time.perf_counter() - t0)
        vals.append(v)
        ones.append(one)
    value = statistics.mean(vals)
    emit({"impl": "reference", "metric": METRIC_C2 if c2 else METRIC, "value": value, "unit": UNIT,
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": "c2_water128_15MeV_e1e6_photon4e6" if c2 else "c4_64_plans_to_1pct",
                     "parallelism": "host cores",
                     "step": "one bounded sample of the workload (below); the rate is per history, so "
                             "it holds for any history count"},
          "extrapolated": False,
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                           "single_core_value": statistics.mean(ones), "cpu_model": cpu_model()},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


def run_c2(args):
    """The paper's timing workload alone (its own JSON line)."""
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
        cpu = oracle_sample_c2()  # spawned processes, before the GPU work starts

    pe, pg = W.config2(W.ELECTRON), W.config2(W.PHOTON)
    nvox = pe.phantom.nvox
    ctx = g.engine(local)
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    pid = ctx.create_phantom(pe.phantom)
    plan_e = ctx.plan_open(pid, pe.source, 1, W_C2)
    plan_g = ctx.plan_open(pid, pg.source, 2, W_C2)
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
    line = {"metric": METRIC_C2, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
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
        line["cpu_baseline"] = {"value": cpu[0], "unit": UNIT, "cores": cpu[2], "kind": "oracle",
                                "sample": cpu[3], "single_core_value": cpu[1], "cpu_model": cpu_model()}
    if rank == 0:
        emit(line)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def c4_seed(spec, rank: int, step: int) -> int:
    """Seed of one plan of the batched workload in a step: every rank and step
    simulates its own, disjoint histories."""
    return (spec.seed + 1_000_003 * (rank + 1) + 7919 * (step + 1000)) % (1 << 62)


def c2_subrecord(ctx, stream, steps: int, warmup: int, rank: int) -> dict:
    """The paper's timing workload (1e6 e- + 4e6 photons at 15 MeV, 128^3
    water at 0.25 cm), each beam from a zeroed tally to FP64 dose and sigma."""
    import torch

    import workloads as W
    pe, pg = W.config2(W.ELECTRON), W.config2(W.PHOTON)
    sh = stream.cuda_stream
    pid = ctx.create_phantom(pe.phantom)
    plan_e = ctx.plan_open(pid, pe.source, 1, W_C2)
    plan_g = ctx.plan_open(pid, pg.source, 2, W_C2)
    d = torch.empty(pe.phantom.nvox, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(d)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(i):
        se = rank_seed(rank, i)
        ctx.plan_reset(plan_e, se, sh)
        ctx.run([plan_e], [N_E], sh)
        a = ctx.plan_result(plan_e, THRESHOLD, d.data_ptr(), sg.data_ptr(), sh)
        ctx.plan_reset(plan_g, se + 1, sh)
        ctx.run([plan_g], [N_G], sh)
        b = ctx.plan_result(plan_g, THRESHOLD, d.data_ptr(), sg.data_ptr(), sh)
        return a, b

    for i in range(warmup):
        step(-1 - i)
    ms, last = [], None
    for i in range(steps):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[0].record(stream)
            last = step(i)
            ev[1].record(stream)
        torch.cuda.synchronize()
        ms.append(ev[0].elapsed_time(ev[1]))
    ctx.plan_close(plan_e)
    ctx.plan_close(plan_g)
    ctx.destroy_phantom(pid)
    a, b = last
    return {"workload": "c2_water128_15MeV_e1e6_photon4e6", "metric": METRIC_C2,
            "value": (N_E + N_G) / (statistics.median(ms) / 1e3), "ms_per_step": statistics.median(ms),
            "steps": steps, "transport_ms_electron": a["transport_ms"], "transport_ms_photon": b["transport_ms"],
            "s05_electron": a["s_thr"], "s05_photon": b["s_thr"],
            "events_electron_beam": a["n_electron_steps"] + a["n_photon_events"],
            "events_photon_beam": b["n_electron_steps"] + b["n_photon_events"],
            "ledger_exact": all(x["e_deposited"] + x["e_escaped"] + x["e_rest"] == x["e_incident"] for x in last)}


def c3_subrecord(ctx, stream, steps: int, warmup: int, rank: int) -> dict:
    """The heterogeneous slab configuration (256^3 at 0.2 cm: water / bone /
    lung / water slabs of 3 / 2 / 6 / rest cm, a 6 MV-like photon spectrum on a
    10x10 cm^2 field), ungrouped and grouped by energy (the same histories and
    bit-identical tallies): its own 1e7 histories from a zeroed tally to FP64
    dose and sigma, then the same plan run from zero to s_0.5 <= 1%."""
    import numpy as np
    import torch

    import workloads as W
    pl = W.config3()
    sh = stream.cuda_stream
    pid = ctx.create_phantom(pl.phantom)
    d = torch.empty(pl.phantom.nvox, dtype=torch.float64, device="cuda")
    sg = torch.empty_like(d)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out, tallies = {}, {}
    for label, grouping in (("ungrouped", W.ENERGY_UNGROUPED), ("grouped", W.ENERGY_GROUPED)):
        pl.source.energy_grouping = grouping
        plan = ctx.plan_open(pid, pl.source, pl.seed, W_C2)

        def step(i):
            ctx.plan_reset(plan, rank_seed(rank, i), sh)
            ctx.run([plan], [pl.n_histories], sh)
            return ctx.plan_result(plan, THRESHOLD, d.data_ptr(), sg.data_ptr(), sh)

        for i in range(warmup):
            step(-1 - i)
        ms, st = [], None
        for i in range(steps):
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[0].record(stream)
                st = step(i)
                ev[1].record(stream)
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        # to 1%: a first round of the configuration's count, then rounds by s ~ 1/sqrt(N)
        ctx.plan_reset(plan, rank_seed(rank, 0), sh)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[0].record(stream)
            r = ctx.run_to_uncertainty([plan], [pl.n_histories], [CAP_C3], TARGET, THRESHOLD, sh)
            ctx.plan_result(plan, THRESHOLD, d.data_ptr(), sg.data_ptr(), sh)
            ev[1].record(stream)
        torch.cuda.synchronize()
        ms1 = ev[0].elapsed_time(ev[1])
        tallies[label] = d.cpu().numpy()
        out[label] = {"value": pl.n_histories / (statistics.median(ms) / 1e3), "ms_per_step": statistics.median(ms),
                      "transport_ms": st["transport_ms"], "s05": st["s_thr"],
                      "ledger_exact": st["e_deposited"] + st["e_escaped"] + st["e_rest"] == st["e_incident"],
                      "to_1pct": {"value": r["histories"][0] / (ms1 / 1e3), "ms": ms1,
                                  "histories": r["histories"][0], "rounds": r["rounds"], "s05": r["s_thr"][0],
                                  "transport_ms": r["transport_ms"]}}
        ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    return {"workload": "c3_slabs256_6MV_photon_1e7", "metric": "histories/s (1e7 photons, 6 MV-like spectrum, "
            "256^3 slabs, to FP64 dose + sigma; and from zero to s_0.5 <= 1%)", "steps": steps, **out,
            "grouped_speedup": out["ungrouped"]["ms_per_step"] / out["grouped"]["ms_per_step"],
            "grouped_speedup_to_1pct": out["ungrouped"]["to_1pct"]["ms"] / out["grouped"]["to_1pct"]["ms"],
            "grouped_dose_equals_ungrouped": bool(np.array_equal(tallies["ungrouped"], tallies["grouped"]))}


def run_c4(args):
    """The contract line: the batched workload's 64 plans, each to s_0.5 <= 1%."""
    import numpy as np
    import torch

    import paper_1101_1245_gb300 as g
    import paper_1101_1245_gb300.roofline as rl
    import workloads as W
    from paper_1101_1245_gb300.autotune import autotune

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample_c4()  # spawned processes, before the GPU work starts

    def log(msg):
        if rank == 0:
            print(f"[bench] {msg}", file=sys.stderr, flush=True)

    specs = W.config4()
    phantoms = c4_phantoms(specs)
    log("phantoms ready")
    ctx = g.engine(local)
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    pids = [ctx.create_phantom(ph) for ph in phantoms]
    srcs = [W.square_field(sp.particle, sp.energy, ph, sp.field_cm) for sp, ph in zip(specs, phantoms)]
    first = [-(-sp.n_histories // W_C4) * W_C4 for sp in specs]
    caps = [CAP_C4] * len(specs)
    # the launch, tuned on the whole plan set at 1/8 of its first round in one launch
    sample = [(pids[i], srcs[i], max(W_C4, first[i] // 8 // W_C4 * W_C4)) for i in range(len(specs))]
    tuned = autotune(ctx, sample, reps=2)
    log(f"autotuned: {tuned['launch']}")
    plans = [ctx.plan_open(pid, src, sp.seed, W_C4) for pid, src, sp in zip(pids, srcs, specs)]

    def seeds(step):
        return [c4_seed(sp, rank, step) for sp in specs]

    def batched(step, target=TARGET):
        for p, sd in zip(plans, seeds(step)):
            ctx.plan_reset(p, sd, sh)
        return ctx.run_to_uncertainty(plans, first, caps, target, THRESHOLD, sh)

    def plain(step, target=TARGET):
        out = {"histories": [], "s_thr": [], "rounds": 0, "transport_ms": 0.0, "sequences": 0}
        for p, sd, f, c in zip(plans, seeds(step), first, caps):
            ctx.plan_reset(p, sd, sh)
            r = ctx.run_to_uncertainty([p], [f], [c], target, THRESHOLD, sh)
            out["histories"] += r["histories"]
            out["s_thr"] += r["s_thr"]
            out["rounds"] += r["rounds"]
            out["transport_ms"] += r["transport_ms"]
            out["sequences"] += r["sequences"]
        return out

    def timed(fn, step):
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            r = fn(step)
            ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), r

    for i in range(args.warmup):
        batched(-1 - i)
    log("warm")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    res = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            res.append(timed(batched, i))
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(sum(r[0] for r in res), dist, dev)
    hist_steps = [sum(r[1]["histories"]) for r in res]
    value = sum(hist_steps) * world / (total_ms / 1e3)
    clocks = clk.summary()
    log(f"batched {value:.3e} histories/s, {total_ms / args.steps:.0f} ms per step")

    # counters of the last timed step: a sequence's event counts go to its first
    # plan, so summing over each type's plans gives that type's sequences
    st = [ctx.plan_result(p, THRESHOLD) for p in plans]
    ev_type = {t: sum(x["n_electron_steps"] + x["n_photon_events"] for x, sp in zip(st, specs) if sp.particle == t)
               for t in (W.ELECTRON, W.PHOTON)}
    last = res[-1][1]
    ledger_ok = all(x["e_deposited"] + x["e_escaped"] + x["e_rest"] == x["e_incident"] for x in st)
    # per plan, n_launches counts the launches of the sequences it ran in (one
    # per round unless a queue overflowed): its folds
    folds = sum(x["n_launches"] for x in st)
    transport_launches = last["sequences"]
    launches = transport_launches + 3 * folds  # + the fold and two s_thr kernels of every fold

    # the plain form: the same plans one at a time, same seeds and schedule
    plain_runs = [timed(plain, i) for i in range(min(2, args.steps))]
    same = all(p[1]["histories"] == res[i][1]["histories"] and p[1]["s_thr"] == res[i][1]["s_thr"]
               for i, p in enumerate(plain_runs))
    plain_value = sum(sum(p[1]["histories"]) for p in plain_runs) / (sum(p[0] for p in plain_runs) / 1e3)
    batched_ms = statistics.median(r[0] for r in res[:len(plain_runs)])
    log(f"plain {plain_value:.3e} histories/s")
    # one round at each plan's own history count (configuration 4 as written):
    # a target every plan meets at once ends the run after its first round
    one = [(timed(lambda i: batched(i, 1e9), 100 + i), timed(lambda i: plain(i, 1e9), 100 + i)) for i in range(3)]
    first_round = {"histories": sum(first), "batched_ms": statistics.median(b[0] for b, _ in one),
                   "plain_ms": statistics.median(p[0] for _, p in one)}
    first_round["batched_over_plain"] = first_round["plain_ms"] / first_round["batched_ms"]
    first_round["batched_value"] = first_round["histories"] / (first_round["batched_ms"] / 1e3)

    # the paper's timing workload, as a sub-record
    for p in plans:
        ctx.plan_close(p)
    c2 = c2_subrecord(ctx, stream, steps=5, warmup=2, rank=rank) if rank == 0 else None
    c3 = c3_subrecord(ctx, stream, steps=5, warmup=2, rank=rank) if rank == 0 else None

    # end to end through the C ABI with host buffers: each step uploads the 64
    # phantoms from pinned host memory, runs them to 1% and reads dose and
    # sigma back into pinned host memory
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    ph_host = [W.Phantom(ph.dims, ph.voxel_cm, pinned(ph.mat), pinned(ph.rho)) for ph in phantoms]
    out_d = [torch.empty(ph.nvox, dtype=torch.float64, pin_memory=True).numpy() for ph in phantoms]
    out_s = [torch.empty(ph.nvox, dtype=torch.float64, pin_memory=True).numpy() for ph in phantoms]

    phases = {}

    def e2e_step(step):
        t = [time.perf_counter()]
        pid2 = [ctx.create_phantom(ph) for ph in ph_host]
        t.append(time.perf_counter())
        pl2 = [ctx.plan_open(pid, src, sd, W_C4) for pid, src, sd in zip(pid2, srcs, seeds(step))]
        t.append(time.perf_counter())
        r = ctx.run_to_uncertainty(pl2, first, caps, TARGET, THRESHOLD)
        t.append(time.perf_counter())
        for p, d, s_ in zip(pl2, out_d, out_s):
            ctx.plan_result_host(p, THRESHOLD, d, s_)
        t.append(time.perf_counter())
        for p in pl2:
            ctx.plan_close(p)
        for pid in pid2:
            ctx.destroy_phantom(pid)
        t.append(time.perf_counter())
        for k, a, b in zip(("create_phantoms", "plan_open", "run_to_uncertainty", "plan_result_host", "close"),
                           t[:-1], t[1:]):
            phases.setdefault(k, []).append(1e3 * (b - a))
        return sum(r["histories"])

    e2e_step(0)  # warm-up (fills the device-memory cache)
    phases.clear()
    e2e = []
    for i in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = e2e_step(i + 1)
        e2e.append(h / (time.perf_counter() - t0))
    e2e_val = statistics.median(e2e) * world
    h2d = sum(ph.mat.nbytes + ph.rho.nbytes for ph in phantoms)
    d2h = sum(16 * ph.nvox for ph in phantoms)
    log(f"e2e {e2e_val:.3e} histories/s")

    served = served_leg(ctx, phantoms, pids, args) if rank == 0 and not args.no_served else None
    if served:
        log(f"served stream {served['stream_value']:.3e} histories/s, p50 {served['latency_p50_s']:.2f} s, "
            f"p99 {served['latency_p99_s']:.2f} s")

    roof = rl.alu_roofline_c4(ev_type[W.ELECTRON], ev_type[W.PHOTON], last["transport_ms"],
                              clocks.get("sm_mhz"), torch.cuda.get_device_properties(dev).multi_processor_count,
                              launches=transport_launches)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4_64_plans_to_1pct",
                       "plans": "64 uneven plans (config 4, seed 4): 64^3-256^3 voxels of 0.2-0.5 cm, "
                                "smoothed-noise densities 0.2-2.0 g/cm^3, 6-18 MeV photon or electron fields "
                                "of 2-15 cm",
                       "target": f"s_0.5 <= {TARGET:g} per plan (mean sigma/D over voxels above 0.5 D_max)",
                       "schedule": "first round = the plan's own history count, then rounds sized by "
                                   "s ~ 1/sqrt(N) (gpumcd_run_to_uncertainty); at most 4e8 histories a plan",
                       "form": "batched: in each round a plan given >= 2^23 histories runs in a launch of its "
                               "own, the others share one launch sequence per particle type (autotuned launch)",
                       "transport_sequences_per_step": last["sequences"],
                       "histories_per_step": statistics.median(hist_steps),
                       "rounds_per_step": last["rounds"],
                       "transport_ms_per_step": last["transport_ms"],
                       "plans_at_cap": sum(1 for h in last["histories"] if h >= CAP_C4),
                       "s_thr_max": max(last["s_thr"]),
                       "n_batches": W_C4,
                       "l2": "inputs larger than L2: 52 GB of batch tallies per step",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "launch": tuned["launch"], "launch_graph": bool(args.graph),
                       "ledger_exact": ledger_ok},
            "plain": {"value": plain_value, "passes": len(plain_runs),
                      "transport_ms_per_step": statistics.median(p[1]["transport_ms"] for p in plain_runs),
                      "transport_sequences_per_step": plain_runs[0][1]["sequences"],
                      "ms_per_step": statistics.median(p[0] for p in plain_runs),
                      "batched_ms_same_seeds": batched_ms,
                      "batched_over_plain": statistics.median(p[0] for p in plain_runs) / batched_ms,
                      "same_histories_and_s_as_batched": same,
                      "form": "each plan alone, the same seeds and schedule (gpumcd_run_to_uncertainty "
                              "with one plan)",
                      "first_round_only": first_round},
            "served": served,
            "c2": c2,
            "c3": c3,
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "host_memory": "pinned", "steps": len(e2e),
                    "form": "64 phantoms uploaded, run to 1% batched, dose and sigma read back, per step",
                    "phases_ms": {k: statistics.median(v) for k, v in phases.items()}},
            "gpu_launches": launches,
            "clocks": clocks}
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": UNIT, "cores": cpu[2], "kind": "oracle",
                                "sample": cpu[3], "single_core_value": cpu[1], "cpu_model": cpu_model()}
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
      MeV electrons), used as listed or stably sorted by decreasing energy:
      two different, equally valid samples of the same dose;
    - a 10x10 cm^2 field whose spectrum (the same energies) is sampled on the
      device, its histories claimed as numbered or in decreasing order of
      energy: the same sample, so on the same kernel the same tally.
    The ungrouped spectrum is also timed on the phase-space kernel that runs
    the grouped one (a same-kernel comparison).  The line reports the share of
    voxels above 10% of the maximum where the two forms agree within 3
    combined sigma."""
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
            # a one-record phase space of the same particle type: run beside a plan
            # (one history), it puts the launch on the phase-space kernel, so the
            # ungrouped spectrum can be timed on the grouped one's kernel too
            rec = np.array([[ph.extent_cm[0] / 2, ph.extent_cm[1] / 2, 0.0, 0.0, 0.0, 1.0, 1.0]])
            dummy = ctx.plan_open(pid, W.Source(particle, W.BEAM_PHASE_SPACE, phase_space=rec), 1, 8)
            out = {}
            forms = [("ungrouped", W.ENERGY_UNGROUPED, False), ("grouped", W.ENERGY_GROUPED, False)]
            if kind == "spectrum":
                forms.insert(1, ("ungrouped_phsp_kernel", W.ENERGY_UNGROUPED, True))
            for label, grouping, with_dummy in forms:
                src.energy_grouping = grouping
                plan = ctx.plan_open(pid, src, pl.seed, 32)

                def once():
                    ctx.plan_reset(plan, pl.seed)
                    ctx.plan_reset(dummy, 1)
                    torch.cuda.synchronize()
                    ev[0].record()
                    if with_dummy:
                        ctx.run([plan, dummy], [pl.n_histories, 1])
                    else:
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
            ctx.plan_close(dummy)
            ctx.destroy_phantom(pid)
            a, b = out["ungrouped"], out["grouped"]
            mask = a["dose"] > 0.1 * a["dose"].max()
            agree = np.abs(a["dose"] - b["dose"]) <= 3.0 * np.sqrt(a["sigma"] ** 2 + b["sigma"] ** 2)
            rows.append({"source": kind, "beam": "electron" if particle == W.ELECTRON else "photon",
                         "histories": pl.n_histories,
                         "transport_ms": {k: v["transport_ms"] for k, v in out.items()},
                         "step_ms": {k: v["ms"] for k, v in out.items()},
                         "grouped_speedup": a["transport_ms"] / b["transport_ms"],
                         "grouped_speedup_same_kernel": (out["ungrouped_phsp_kernel"]["transport_ms"]
                                                         / b["transport_ms"]) if kind == "spectrum" else
                         a["transport_ms"] / b["transport_ms"],
                         "electron_steps_per_history": {k: v["electron_steps_per_history"] for k, v in out.items()},
                         "ledger_exact": all(v["ledger_exact"] for v in out.values()),
                         "dose_3sigma_agreement": float(agree[mask].mean())})
    ctx.close()
    emit({"workload": "polyenergetic_energy_grouping_c2_phantom",
          "metric": "transport ms per beam, ungrouped vs grouped by energy",
          "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
          "phantom": "128^3 water at 0.25 cm", "data": "synthetic", "rows": rows})


def served_leg(ctx, phantoms, pids, args) -> dict:
    """Config 5: a Poisson stream of dose requests from the config-4
    distribution on resident phantoms (request i on phantom i mod 64), served
    with continuous batching to s_0.5 <= target; first a capacity run of a
    calibration set all present at once, against the same requests run one by
    one with the plain schedule (serve.run_alone), then the stream at 0.8 x that
    capacity."""
    import workloads as W
    from paper_1101_1245_gb300.serve import DoseRequest, Server, run_alone

    budget = int(args.budget_gb * 2 ** 30)

    def requests(rate):
        reqs = []
        for i, r in enumerate(W.config5(count=args.requests, rate_per_s=rate)):
            k = i % len(phantoms)
            ph, sp = phantoms[k], r.spec
            src = W.square_field(sp.particle, sp.energy, ph, sp.field_cm)
            reqs.append(DoseRequest(i, pids[k], ph.nvox, src, sp.seed, r.arrival_s, CAP_C4))
        return reqs

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
    srv = Server(ctx, budget, target=args.target, round_histories=args.round_histories,
                 rounds_in_flight=args.rounds_in_flight)
    for q in requests(rate):
        srv.submit(q)
    results = srv.run(real_time=True)
    rep = srv.report()
    # the same stream served first come first served, each request alone at the
    # measured alone rate (a model from the requests' histories, not a run):
    # what continuous batching changes in latency at the same throughput
    import numpy as np
    alone_rate = alone_h / alone_t if alone_t else None
    fifo = None
    if alone_rate:
        t_free, lat = 0.0, []
        for r in sorted(results, key=lambda r: r.arrival_s):
            start = max(t_free, r.arrival_s)
            t_free = start + r.histories / alone_rate
            lat.append(t_free - r.arrival_s)
        fifo = {"latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "basis": "each request's histories at the measured alone rate, in arrival order"}
    return {"target": args.target, "threshold": THRESHOLD,
            "capacity_value": rep_cal["histories_per_s"],
            "alone_value": alone_h / alone_t if alone_t else None,
            "served_over_alone": rep_cal["histories_per_s"] * alone_t / alone_h if alone_h else None,
            "capacity_requests": len(cal), "capacity_histories": rep_cal["histories"],
            "alone_histories": alone_h, "capacity_rounds": rep_cal["rounds"],
            "requests": rep["requests"], "arrival_rate_per_s": rate,
            "rate_basis": "0.8 x the served capacity on the calibration set",
            "stream_value": rep["histories_per_s"], "latency_p50_s": rep["latency_p50_s"],
            "latency_p99_s": rep["latency_p99_s"], "fifo_alone_model": fifo,
            "wall_s": rep["wall_s"], "rounds": rep["rounds"],
            "folds": rep["folds"], "mean_histories_per_request": rep["histories"] / max(rep["requests"], 1),
            "s_thr_max": rep["s_thr_max"], "rounds_in_flight": args.rounds_in_flight,
            "round_histories": args.round_histories, "hbm_budget_gb": args.budget_gb,
            "max_histories_per_request": CAP_C4,
            "phantoms": "64 resident config-4 phantoms, request i on phantom i mod 64"}


def run_served(args):
    import paper_1101_1245_gb300 as g
    import workloads as W

    phantoms = c4_phantoms(W.config4())
    ctx = g.engine(0, hbm_budget_bytes=int(args.budget_gb * 2 ** 30) + (8 << 30))
    if args.graph:
        ctx.set_launch(flags=g.LAUNCH_GRAPH)
    pids = [ctx.create_phantom(ph) for ph in phantoms]
    out = served_leg(ctx, phantoms, pids, args)
    emit({"workload": "c5_served", "metric": "histories/s and request latency at s_0.5 <= target",
          "unit": UNIT, **out, "launch_graph": bool(args.graph), "data": "synthetic"})
    ctx.close()


def run_ncu_case(args):
    """A small case of the workload for ncu, untimed.  c2: each beam once at 1/5
    of its histories (one transport launch per beam).  c4: the batched
    workload's plans of at most 160^3 voxels (8 batch tallies each, a few GB on
    the device), one round at 1/10 of their first-round histories: one
    transport launch per particle type.  Prints each launch's event counts."""
    import paper_1101_1245_gb300 as g
    import workloads as W

    ctx = g.engine(0)
    if args.workload == "c4":
        specs = [sp for sp in W.config4() if sp.n <= 160]
        phantoms = c4_phantoms(specs)
        pids = [ctx.create_phantom(ph) for ph in phantoms]
        for t in (W.ELECTRON, W.PHOTON):
            idx = [i for i, sp in enumerate(specs) if sp.particle == t]
            plans = [ctx.plan_open(pids[i], W.square_field(specs[i].particle, specs[i].energy, phantoms[i],
                                                           specs[i].field_cm), specs[i].seed, 8) for i in idx]
            n = [max(8, specs[i].n_histories // 10 // 8 * 8) for i in idx]
            ctx.run(plans, n)
            st = [ctx.plan_result(p, 0.5) for p in plans]
            print(json.dumps({"case": "c4_small_" + ("electron" if t == W.ELECTRON else "photon"),
                              "plans": len(plans), "histories": sum(n),
                              "voxels": int(sum(phantoms[i].nvox for i in idx)),
                              **{k: sum(x[k] for x in st) for k in (
                                  "n_electron_steps", "n_photon_events", "n_hard_real")},
                              "n_launches": st[0]["n_launches"], "transport_ms": st[0]["transport_ms"]}),
                  flush=True)
            for p in plans:
                ctx.plan_close(p)
        ctx.close()
        return
    for part, n in ((W.ELECTRON, N_E // 5), (W.PHOTON, N_G // 5)):
        pl = W.config2(part)
        pid = ctx.create_phantom(pl.phantom)
        plan = ctx.plan_open(pid, pl.source, 5, W_C2)
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
        run_ncu_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run = {"c4": run_c4, "c2": run_c2, "batched": run_batched, "served": run_served, "geoms": run_geoms,
           "ablation": run_ablation, "kerma": run_kerma, "grouping": run_grouping}
    run[args.workload](args)


if __name__ == "__main__":
    main()

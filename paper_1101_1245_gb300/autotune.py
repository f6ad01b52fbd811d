"""Launch autotuner for the persistent transport kernel.

The kernel's launch shape (threads per CTA, resident CTAs per SM) and its
scheduling knobs (primaries claimed per chunk, the stack level at which a warp
switches particle type, the lane count below which it switches) change its
speed but never its result: every particle's random stream and energy ledger
are independent of scheduling, so the tally is bit-identical for any setting.
The tuner therefore times real plans - a sample of the workload at reduced
history counts - under candidate settings by coordinate descent and keeps the
fastest.  A setting the library refuses for the sampled plans (the
phase-space kernel, which also draws grouped spectra, runs at most two CTAs
per SM) is recorded as a refused trial and skipped, and so is a setting under
which the particle queues overflow (a switch level close to the stack
capacity spills most stacked particles).
"""
from __future__ import annotations

import statistics
from typing import Dict, List, Sequence, Tuple

from . import ERR_INVALID_ARG, ERR_QUEUE_OVERFLOW, Context, GpumcdError

# (block_threads, blocks_per_sm) shapes with a kernel variant behind them: 32
# warps per SM in one CTA (64 registers, one copy of the tables per SM) or two,
# 24 warps (80 registers), 16 warps (128 registers)
SHAPES: List[Tuple[int, int]] = [(1024, 1), (512, 2), (384, 2), (256, 3), (512, 1)]
KNOBS: Dict[str, List[int]] = {
    "chunk": [16, 32, 64],
    "switch_high": [200, 320, 384],
    "refill_low": [8, 16, 24],
}


def _time(ctx: Context, plans: Sequence[int], hist: Sequence[int], reps: int) -> float:
    ts = []
    for r in range(reps):
        for p in plans:
            ctx.plan_reset(p, 1000 + r)
        ctx.run(plans, hist)
        ts.append(ctx.plan_result(plans[0], 0.5)["transport_ms"])
    return statistics.median(ts)


def _try(ctx: Context, plans, hist, reps: int):
    """Transport ms under the launch set on ctx, or None if the library refuses
    that launch for these plans or its particle queues overflow under it (the
    run then stops with an error status and marks the plans failed; the next
    trial resets them)."""
    try:
        return _time(ctx, plans, hist, reps)
    except GpumcdError as e:
        if e.status not in (ERR_INVALID_ARG, ERR_QUEUE_OVERFLOW):
            raise
        return None


def autotune(ctx: Context, samples: Sequence[Tuple[int, object, int]], reps: int = 3,
             n_batches: int = 16) -> dict:
    """samples: (phantom_id, workload Source, histories) triples run together in
    one batched launch per trial.  Leaves the best launch on ctx and returns it
    with the trial timings (ms of transport per trial; None for a launch the
    library refused)."""
    plans = [ctx.plan_open(pid, src, 1, n_batches) for pid, src, _ in samples]
    hist = [n for _, _, n in samples]
    base = ctx.get_launch()
    trials = []
    try:
        best = dict(base)
        best_ms = None
        for bt, bps in SHAPES:
            cand = dict(best, block_threads=bt, blocks_per_sm=bps,
                        stack_capacity=max(best["stack_capacity"], 512))
            ctx.set_launch(**cand)
            ms = _try(ctx, plans, hist, reps)
            trials.append((dict(block_threads=bt, blocks_per_sm=bps), ms))
            if ms is not None and (best_ms is None or ms < best_ms):
                best, best_ms = cand, ms
        if best_ms is None:
            ctx.set_launch(**base)
            raise GpumcdError(ERR_INVALID_ARG, "autotune: every launch shape refused")
        for knob, values in KNOBS.items():
            for v in values:
                if v == best[knob]:
                    continue
                cand = dict(best, **{knob: v})
                if cand["switch_high"] > cand["stack_capacity"]:
                    continue
                ctx.set_launch(**cand)
                ms = _try(ctx, plans, hist, reps)
                trials.append(({knob: v}, ms))
                if ms is not None and ms < best_ms:
                    best, best_ms = cand, ms
        ctx.set_launch(**best)
    finally:
        for p in plans:
            ctx.plan_close(p)
    return {"launch": best, "transport_ms": best_ms, "trials": trials}

"""Dose-calculation serving loop: continuous batching over the gpumcd C ABI.

Requests (a resident phantom, a beam, a seed) arrive over time.  The server
admits them as plans while the HBM budget allows, and runs the active plans in
rounds: each round is one batched persistent launch sequence over the plans
that still have work before their next fold, each simulating its next chunk
of histories.  Up to ``MAX_INFLIGHT`` rounds are on the device at once
(gpumcd_submit), so one round's CTAs fill the SMs that the other round's drain
frees.  A plan's tally is folded (FP64, on the device) when it reaches the
history count at which its uncertainty was projected to reach the target and
none of its histories is in flight; a plan whose relative uncertainty s (mean
sigma/D over voxels above ``threshold`` x D_max, GPUMCD §II.D) has reached
``target`` is retired: its dose is returned and its tally memory freed.  New
arrivals join the next round, so work from requests that arrived at different
times overlaps on the device.

A plan's histories are numbered from 0 in submission order and its random
streams depend only on (seed, history, lineage, draw), so its result after N
histories is the same bit for bit whether it ran alone or in any mix, in any
chunking, with any overlap.
"""
from __future__ import annotations

import collections
import dataclasses
import heapq
import math
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import Context, GpumcdError, MAX_INFLIGHT, MAX_PLANS_PER_RUN


@dataclasses.dataclass
class DoseRequest:
    """One dose calculation: a resident phantom id, a workload Source, a seed."""

    rid: int
    phantom_id: int
    nvox: int
    source: object
    seed: int
    arrival_s: float = 0.0
    max_histories: int = 2_000_000_000


@dataclasses.dataclass
class DoseResult:
    rid: int
    histories: int
    s_thr: float
    arrival_s: float
    admitted_s: float
    done_s: float
    rounds: int
    dose: Optional[np.ndarray] = None
    sigma: Optional[np.ndarray] = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclasses.dataclass
class _Active:
    req: DoseRequest
    plan: int
    admitted_s: float
    bytes: int
    histories: int = 0   # histories of finished rounds
    submitted: int = 0   # histories handed to rounds (finished or in flight)
    inflight: int = 0    # rounds in flight that include the plan
    s_thr: float = float("inf")
    rounds: int = 0
    next_check: int = 0  # history count at which the tally is next folded


class Server:
    """Continuous-batching dose server on one gpumcd context.

    target        relative uncertainty s at which a plan is retired
    threshold     dose fraction of D_max above which s is averaged (0.5 here)
    n_batches     batch tallies per plan (the sigma estimator)
    round_histories  histories per round over all active plans
    first_chunk   histories of a new plan's first round
    hbm_budget    bytes of tallies the server may hold at once
    rounds_in_flight  rounds on the device at once (1 .. MAX_INFLIGHT)
    stagger_first     first checkpoints at 1, 2 or 3 first chunks by request id
    """

    def __init__(self, ctx: Context, hbm_budget: int, target: float = 0.01,
                 threshold: float = 0.5, n_batches: int = 16,
                 round_histories: int = 16_000_000, first_chunk: int = 200_000,
                 keep_dose: bool = False, clock: Callable[[], float] = time.perf_counter,
                 rounds_in_flight: int = MAX_INFLIGHT, stagger_first: bool = True,
                 log_rounds: bool = False):
        self.ctx = ctx
        self.budget = hbm_budget
        self.target = target
        self.threshold = threshold
        self.W = n_batches
        self.round_histories = round_histories
        self.first_chunk = first_chunk
        self.keep_dose = keep_dose
        self.clock = clock
        if not 1 <= rounds_in_flight <= MAX_INFLIGHT:
            raise ValueError(f"rounds_in_flight must be in [1, {MAX_INFLIGHT}]")
        self.depth = rounds_in_flight
        self.stagger = stagger_first
        # with log_rounds: (plans, histories, submitted_s, finished_s) per round
        self.round_log: Optional[List[tuple]] = [] if log_rounds else None
        self.used = 0
        self.waiting: List[tuple] = []  # heap of (arrival, rid, request)
        self.active: Dict[int, _Active] = {}
        self.results: List[DoseResult] = []
        self.total_histories = 0
        self.rounds = 0
        self._turn = 0
        self.max_active = 0
        self.max_used = 0
        self.folds = 0
        self.inflight: collections.deque = collections.deque()  # (ticket, [(plan, histories)], submitted_s)
        self.t0 = None

    # ---- requests ------------------------------------------------------
    def tally_bytes(self, req: DoseRequest) -> int:
        return self.W * req.nvox * 8 + 64

    def submit(self, req: DoseRequest) -> None:
        if self.tally_bytes(req) > self.budget:
            raise GpumcdError(-7, "request larger than the HBM budget")
        heapq.heappush(self.waiting, (req.arrival_s, req.rid, req))

    # ---- scheduling -----------------------------------------------------
    def _now(self) -> float:
        return self.clock() - self.t0

    def _admit(self) -> None:
        now = self._now()
        while (self.waiting and self.waiting[0][0] <= now
               and len(self.active) < MAX_PLANS_PER_RUN):
            req = self.waiting[0][2]
            need = self.tally_bytes(req)
            if self.used + need > self.budget:
                break  # wait for memory to free up (requests stay in arrival order)
            heapq.heappop(self.waiting)
            plan = self.ctx.plan_open(req.phantom_id, req.source, req.seed, self.W)
            self.active[plan] = _Active(req, plan, now, need)
            self.used += need
            self.max_active = max(self.max_active, len(self.active))
            self.max_used = max(self.max_used, self.used)

    def _quantum(self) -> int:
        # chunks are whole multiples of W histories (history h goes to batch
        # h mod W), so every batch holds the same number of histories and the
        # fold takes its exact-integer form
        return self.W

    def _chunk(self, a: _Active, share: int) -> int:
        """Histories for a plan's next round: its first chunk, then up to the
        point where its tally is next folded, within its share of the round."""
        q = self._quantum()
        if a.submitted == 0:
            # first checkpoints at 1, 2 or 3 first chunks (by request id): requests
            # that arrive together then reach their folds at different rounds, so
            # the device is not idle while all of them fold at once
            a.next_check = self.first_chunk * (1 + a.req.rid % 3 if self.stagger else 1)
        n = min(a.next_check - a.submitted, share)
        n = max(q, -(-n // q) * q)
        return int(max(1, min(n, a.req.max_histories - a.submitted)))

    def _runnable(self) -> List[_Active]:
        return [a for a in self.active.values()
                if a.submitted < max(a.next_check, 1) and a.submitted < a.req.max_histories]

    @staticmethod
    def _kind(a: "_Active") -> int:
        return int(getattr(a.req.source, "particle", 0))

    def _submit_rounds(self) -> None:
        """Fill the free launch slots with rounds over the plans that have work.
        A round carries one particle type, the types taking turns: a launch that
        draws electron and photon primaries at once is slower (its warps switch
        type far more often), and with two rounds in flight both types still run
        together, each in its own launch."""
        while len(self.inflight) < self.depth:
            plans = self._runnable()
            if not plans:
                return
            kinds = sorted({self._kind(a) for a in plans})
            if len(kinds) > 1:
                k = kinds[self._turn % len(kinds)]
                self._turn += 1
                plans = [a for a in plans if self._kind(a) == k]
            share = max(self.round_histories // len(plans), self._quantum())
            chunks = [self._chunk(a, share) for a in plans]
            ticket = self.ctx.submit([a.plan for a in plans], chunks)
            for a, n in zip(plans, chunks):
                a.submitted += n
                a.inflight += 1
            self.inflight.append((ticket, list(zip(plans, chunks)), self._now()))
            self.rounds += 1

    def _finish_oldest(self) -> None:
        ticket, pairs, t_sub = self.inflight.popleft()
        self.ctx.wait(ticket)
        if self.round_log is not None:
            self.round_log.append((len(pairs), sum(n for _, n in pairs), t_sub, self._now()))
        for a, n in pairs:
            a.histories += n
            a.inflight -= 1
            a.rounds += 1
            self.total_histories += n

    def _fold_ready(self) -> None:
        """Fold every plan at its checkpoint with no histories in flight."""
        for a in list(self.active.values()):
            if a.inflight or a.submitted == 0:
                continue
            if a.histories < a.next_check and a.histories < a.req.max_histories:
                continue
            self.folds += 1
            if self.keep_dose:
                import torch
                d = torch.empty(a.req.nvox, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
                s = torch.empty_like(d)
                st = self.ctx.plan_result(a.plan, self.threshold, d.data_ptr(), s.data_ptr())
            else:
                st = self.ctx.plan_result(a.plan, self.threshold)
            a.s_thr = st["s_thr"] if st["s_thr"] > 0 else float("inf")
            if a.s_thr <= self.target or a.histories >= a.req.max_histories:
                res = DoseResult(a.req.rid, a.histories, a.s_thr, a.req.arrival_s, a.admitted_s,
                                 self._now(), a.rounds)
                if self.keep_dose:
                    res.dose, res.sigma = d.cpu().numpy(), s.cpu().numpy()
                self.results.append(res)
                self.ctx.plan_close(a.plan)
                self.used -= a.bytes
                del self.active[a.plan]
            else:
                # s ~ 1/sqrt(N): the history count expected to reach the target,
                # with 5% to spare, and at least 10% more than now
                a.next_check = int(max(a.histories * (a.s_thr / self.target) ** 2 * 1.05,
                                       a.histories * 1.1))

    def run(self, real_time: bool = True) -> List[DoseResult]:
        """Serves every submitted request.  With real_time, requests become
        visible at their arrival times on the server clock; otherwise all at once."""
        self.t0 = self.clock()
        self.inflight = collections.deque()
        if not real_time:
            self.waiting = [(0.0, r, q) for (_, r, q) in self.waiting]
            heapq.heapify(self.waiting)
        try:
            while self.waiting or self.active or self.inflight:
                self._admit()
                self._submit_rounds()
                if not self.inflight:
                    before = len(self.active)
                    self._fold_ready()
                    if self.active and len(self.active) == before and not self._runnable():
                        raise RuntimeError("served plans stalled")  # cannot happen: folds move next_check
                    if not self.active and self.waiting:
                        dt = self.waiting[0][0] - self._now()
                        if dt > 0:
                            time.sleep(min(dt, 0.05))
                    continue
                self._finish_oldest()
                # keep the device busy before blocking on folds
                self._admit()
                self._submit_rounds()
                self._fold_ready()
        finally:
            while self.inflight:  # leave no sequence in flight on an error
                ticket = self.inflight.popleft()[0]
                try:
                    self.ctx.wait(ticket)
                except GpumcdError:
                    pass
        return self.results

    # ---- reporting ----------------------------------------------------------
    def report(self) -> dict:
        lat = np.array([r.latency_s for r in self.results])
        wall = self._now() if self.t0 is not None else 0.0
        return {
            "requests": len(self.results),
            "histories": int(self.total_histories),
            "wall_s": wall,
            "histories_per_s": self.total_histories / wall if wall > 0 else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "rounds": self.rounds,
            "folds": self.folds,
            "s_thr_max": float(max(r.s_thr for r in self.results)) if self.results else None,
        }


def run_alone(ctx: Context, req: DoseRequest, target: float, threshold: float = 0.5,
              n_batches: int = 16, first_chunk: int = 200_000) -> DoseResult:
    """The plain form: one request run by itself to the target with the same
    schedule as the server (a first chunk, then runs up to the projected
    history count, folding the tally after each run)."""
    t0 = time.perf_counter()
    q = n_batches
    plan = ctx.plan_open(req.phantom_id, req.source, req.seed, n_batches)
    done, rounds, s = 0, 0, float("inf")
    try:
        goal = first_chunk
        while True:
            n = max(q, -(-(goal - done) // q) * q)
            n = max(1, min(n, req.max_histories - done))
            ctx.run([plan], [n])
            done += n
            rounds += 1
            st = ctx.plan_result(plan, threshold)
            s = st["s_thr"] if st["s_thr"] > 0 else float("inf")
            if s <= target or done >= req.max_histories:
                break
            goal = int(max(done * (s / target) ** 2 * 1.05, done * 1.1))
    finally:
        ctx.plan_close(plan)
    t1 = time.perf_counter()
    return DoseResult(req.rid, done, s, 0.0, 0.0, t1 - t0, rounds)

"""Host logic of the continuous-batching server, against a fake context that
keeps the C ABI's rules (no GPU): at most MAX_INFLIGHT sequences, no result,
reset or close of a plan that is in a sequence still in flight, histories
numbered in submission order.  The fake's relative uncertainty of a plan
after N histories is c / sqrt(N), the 1/sqrt(N) law of §II.D."""
import math

import pytest

import paper_1101_1245_gb300 as g
from paper_1101_1245_gb300.serve import DoseRequest, Server, run_alone


class FakeCtx:
    device = 0

    def __init__(self, coef):
        self.coef = coef          # phantom id -> c in s = c / sqrt(N)
        self.plans = {}
        self.next_plan = 1
        self.next_ticket = 1
        self.tickets = {}         # ticket -> [(plan, n)]
        self.max_inflight = 0
        self.chunks = []
        self.log = []

    def plan_open(self, pid, src, seed, W):
        p = self.next_plan
        self.next_plan += 1
        self.plans[p] = {"pid": pid, "W": W, "sub": 0, "done": 0, "inflight": 0}
        return p

    def _busy(self, p):
        if self.plans[p]["inflight"]:
            raise g.GpumcdError(g.ERR_STATE, "plan in flight")

    def plan_close(self, p):
        self._busy(p)
        del self.plans[p]

    def submit(self, plans, ns):
        if len(self.tickets) >= g.MAX_INFLIGHT:
            raise g.GpumcdError(g.ERR_STATE, "gpumcd_submit")
        assert len(plans) <= g.MAX_PLANS_PER_RUN and len(set(plans)) == len(plans)
        for p, n in zip(plans, ns):
            st = self.plans[p]
            assert n > 0 and n % st["W"] == 0
            self.log.append((p, st["sub"], n))
            st["sub"] += n
            st["inflight"] += 1
            self.chunks.append(n)
        t = self.next_ticket
        self.next_ticket += 1
        self.tickets[t] = list(zip(plans, ns))
        self.max_inflight = max(self.max_inflight, len(self.tickets))
        return t

    def wait(self, t):
        for p, n in self.tickets.pop(t):
            self.plans[p]["inflight"] -= 1
            self.plans[p]["done"] += n

    def run(self, plans, ns):
        self.wait(self.submit(plans, ns))

    def plan_result(self, p, thr, d=0, s=0):
        self._busy(p)
        st = self.plans[p]
        return {"s_thr": self.coef[st["pid"]] / math.sqrt(st["done"]), "histories": st["done"]}


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4
        return self.t


def _requests(n, nvox=1000):
    return [DoseRequest(i, i % 5, nvox, None, 100 + i, arrival_s=0.0) for i in range(n)]


def test_every_request_reaches_the_target():
    coef = {k: 2.0 + k for k in range(5)}
    ctx = FakeCtx(coef)
    srv = Server(ctx, hbm_budget=1 << 40, target=0.01, n_batches=16, round_histories=200_000,
                 first_chunk=10_000, clock=Clock())
    for r in _requests(30):
        srv.submit(r)
    res = srv.run(real_time=False)
    assert sorted(r.rid for r in res) == list(range(30))
    for r in res:
        need = (coef[r.rid % 5] / 0.01) ** 2
        assert r.s_thr <= 0.01 and r.histories >= need
        # the projection overshoots by at most its 5% margin (+ one quantum and a first chunk)
        assert r.histories <= 1.2 * need + 10_016
    assert ctx.max_inflight == g.MAX_INFLIGHT
    assert not ctx.tickets and not ctx.plans and srv.used == 0
    assert all(n % 16 == 0 for n in ctx.chunks)


def test_histories_are_numbered_in_submission_order():
    ctx = FakeCtx({k: 3.0 for k in range(5)})
    srv = Server(ctx, hbm_budget=1 << 40, target=0.02, round_histories=50_000, first_chunk=4_000,
                 clock=Clock())
    for r in _requests(8):
        srv.submit(r)
    srv.run(real_time=False)
    by_plan = {}
    for p, base, n in ctx.log:
        assert base == by_plan.get(p, 0)  # contiguous, no gaps or overlaps
        by_plan[p] = base + n


def test_budget_and_plan_limits():
    ctx = FakeCtx({k: 2.0 for k in range(5)})
    one = 16 * 1000 * 8 + 64
    srv = Server(ctx, hbm_budget=3 * one, target=0.02, round_histories=100_000, first_chunk=5_000,
                 clock=Clock())
    for r in _requests(12):
        srv.submit(r)
    res = srv.run(real_time=False)
    assert len(res) == 12
    assert srv.max_used <= 3 * one and srv.max_active == 3
    with pytest.raises(g.GpumcdError):
        srv.submit(DoseRequest(99, 0, 10 ** 9, None, 1))


def test_alone_follows_the_same_schedule():
    ctx = FakeCtx({0: 2.5})
    r = run_alone(ctx, DoseRequest(0, 0, 1000, None, 7), target=0.01, first_chunk=10_000)
    assert r.s_thr <= 0.01 and r.histories >= (2.5 / 0.01) ** 2
    assert all(n % 16 == 0 for n in ctx.chunks)


def test_rounds_carry_one_particle_type_in_turn():
    """A round holds plans of one particle type, the types taking turns, and
    every request of either type still reaches the target."""
    import types
    ctx = FakeCtx({k: 2.0 for k in range(5)})
    rounds = []
    submit = ctx.submit

    def spy(plans, ns):
        rounds.append(list(plans))
        return submit(plans, ns)

    ctx.submit = spy
    srv = Server(ctx, hbm_budget=1 << 40, target=0.02, round_histories=100_000, first_chunk=5_000,
                 clock=Clock())
    kind = {}
    for i in range(10):
        src = types.SimpleNamespace(particle=i % 2)
        r = DoseRequest(i, i % 5, 1000, src, 100 + i)
        srv.submit(r)
        kind[i] = i % 2
    res = srv.run(real_time=False)
    assert sorted(r.rid for r in res) == list(range(10))
    # plans open in admission order, which is request order here (the budget admits all)
    opened = sorted({p for rnd in rounds for p in rnd})
    plan_kind = {p: kind[rid] for rid, p in enumerate(opened)}
    mixed = [rnd for rnd in rounds if len({plan_kind[p] for p in rnd}) > 1]
    assert not mixed
    assert {plan_kind[rounds[0][0]], plan_kind[rounds[1][0]]} == {0, 1}  # the types alternate

"""Host logic of the launch autotuner, against a fake context (no GPU): it
keeps the fastest launch, skips the launches the library refuses for the
sampled plans (as it refuses more than two CTAs per SM to the phase-space
kernel), and closes its plans whatever happens."""
import pytest

import paper_1101_1245_gb300 as g
from paper_1101_1245_gb300.autotune import autotune


class FakeCtx:
    def __init__(self, cost, refuse):
        self.launch = {"block_threads": 512, "blocks_per_sm": 2, "stack_capacity": 512,
                       "switch_high": 320, "refill_low": 16, "chunk": 32}
        self.cost, self.refuse = cost, refuse
        self.open, self.next_id, self.last_ms = set(), 0, None

    def plan_open(self, pid, src, seed, n_batches):
        self.next_id += 1
        self.open.add(self.next_id)
        return self.next_id

    def plan_close(self, p):
        self.open.remove(p)

    def plan_reset(self, p, seed):
        pass

    def get_launch(self):
        return dict(self.launch)

    def set_launch(self, **kw):
        self.launch.update(kw)

    def run(self, plans, hist):
        if self.refuse(self.launch):
            raise g.GpumcdError(g.ERR_INVALID_ARG, "gpumcd_run")
        self.last_ms = self.cost(self.launch)

    def plan_result(self, p, thr):
        return {"transport_ms": self.last_ms}


def _cost(L):
    # fastest at 256 x 3 with chunk 64; every other knob costs a little
    return (abs(L["blocks_per_sm"] - 3) + abs(L["block_threads"] - 256) / 100 + (64 - L["chunk"]) / 10
            + abs(L["switch_high"] - 320) / 1000 + abs(L["refill_low"] - 16) / 1000 + 1.0)


def test_autotune_keeps_the_fastest_launch():
    ctx = FakeCtx(_cost, lambda L: False)
    res = autotune(ctx, [(0, None, 100), (1, None, 200)], reps=1)
    assert res["launch"]["block_threads"] == 256 and res["launch"]["blocks_per_sm"] == 3
    assert res["launch"]["chunk"] == 64
    assert ctx.launch == res["launch"] and not ctx.open


def test_autotune_skips_refused_launches():
    ctx = FakeCtx(_cost, lambda L: L["blocks_per_sm"] > 2)
    res = autotune(ctx, [(0, None, 100)], reps=1)
    assert res["launch"]["blocks_per_sm"] <= 2
    refused = [t for t in res["trials"] if t[1] is None]
    assert refused == [({"block_threads": 256, "blocks_per_sm": 3}, None)]
    assert ctx.launch == res["launch"] and not ctx.open


def test_autotune_refused_everywhere_restores_the_launch():
    ctx = FakeCtx(_cost, lambda L: True)
    before = ctx.get_launch()
    with pytest.raises(g.GpumcdError) as e:
        autotune(ctx, [(0, None, 100)], reps=1)
    assert e.value.status == g.ERR_INVALID_ARG
    assert ctx.launch == before and not ctx.open


def test_autotune_skips_settings_that_overflow_the_queues():
    """A setting under which a trial run stops with a queue overflow (an error
    status, nothing dropped) is recorded as refused; the tuner goes on."""
    def run(plans, hist):
        if ctx.launch["switch_high"] >= 384:
            raise g.GpumcdError(g.ERR_QUEUE_OVERFLOW, "gpumcd_run")
        ctx.last_ms = _cost(ctx.launch)

    ctx = FakeCtx(_cost, lambda L: False)
    ctx.run = run
    res = autotune(ctx, [(0, None, 100)], reps=1)
    assert res["launch"]["switch_high"] < 384
    assert ({"switch_high": 384}, None) in res["trials"]
    assert ctx.launch == res["launch"] and not ctx.open


def test_autotune_passes_other_errors_on():
    def boom(L):
        raise g.GpumcdError(g.ERR_CUDA, "gpumcd_run")

    ctx = FakeCtx(_cost, lambda L: False)
    ctx.run = lambda plans, hist: boom(ctx.launch)
    with pytest.raises(g.GpumcdError) as e:
        autotune(ctx, [(0, None, 100)], reps=1)
    assert e.value.status == g.ERR_CUDA and not ctx.open

"""Fixtures and helpers for the GPU tests (imports the CUDA binding lazily)."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.conftest import host_cores


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make_ctx(**launch):
    import paper_1101_1245_gb300 as g
    need_gpu()
    ctx = g.engine(0)
    if launch:
        ctx.set_launch(**launch)
    return ctx


def run_gpu(ctx, plan, n=None, seed=None):
    pid = ctx.create_phantom(plan.phantom)
    try:
        r = ctx.simulate(pid, plan.source, n or plan.n_histories,
                         plan.seed if seed is None else seed, nvox=plan.phantom.nvox)
    finally:
        ctx.destroy_phantom(pid)
    return r


def run_oracle(plan, n=None, seed=None, flags=0, mats=None):
    return oracle.simulate(mats if mats is not None else W.MATERIALS, W.DEFAULT_PHYSICS, plan.phantom, plan.source,
                           n or plan.n_histories, plan.seed if seed is None else seed, flags,
                           processes=host_cores())


def ledger_exact(stats) -> bool:
    return stats["e_deposited"] + stats["e_escaped"] + stats["e_rest"] == stats["e_incident"]

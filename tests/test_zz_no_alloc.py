"""The allocation-free result call against the regular one.

gpumcd_plan_result_noalloc exists for callers that cannot allocate device
memory when they fetch a result (a serving loop whose HBM budget is fully
committed, or a latency-bound loop where cudaMalloc/cudaFree would stall the
device).  It folds the same tally with its scratch in a fixed device array.
This file is collected last so that a failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import paper_1101_1245_gb300 as g
import workloads as W
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu


def _noalloc(ctx, plan, dose, sigma):
    st = g.RunStats()
    status = g.lib().gpumcd_plan_result_noalloc(ctx.h, plan, 0.5, dose.data_ptr(), sigma.data_ptr(),
                                                None, ctypes.byref(st))
    return status, st.as_dict()


@pytest.mark.parametrize("n_batches", [8, 16, 32, 64])
def test_noalloc_result_matches_plan_result_twice(n_batches):
    """Two calls in a row on one plan, each against gpumcd_plan_result: the
    first after 30,005 histories (unequal batches: the two-pass FP64 form),
    the second after 40,000 (equal batches: the integer-variance form).  Both
    calls use the regular fold's per-voxel arithmetic, so dose and sigma are
    equal bit for bit; s_thr sums in another order (relative 1e-12)."""
    import torch
    ctx = make_ctx()
    ph = W.z_slabs((40, 36, 48), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                        (5.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    pid = ctx.create_phantom(ph)
    src = W.Source(W.ELECTRON, W.BEAM_SQUARE, energy=9.0, center_cm=(10.0, 9.0), field_cm=6.0)
    plan = ctx.plan_open(pid, src, 21, n_batches)
    ctx.run([plan], [30_005])
    d_ref = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s_ref = torch.zeros_like(d_ref)
    ref = ctx.plan_result(plan, 0.5, d_ref.data_ptr(), s_ref.data_ptr())
    used_before = ctx.memory()[0]
    for call in range(2):
        d = torch.full_like(d_ref, -1.0)
        s = torch.full_like(d_ref, -1.0)
        status, st = _noalloc(ctx, plan, d, s)
        assert status == g.OK, g.status_string(status)
        assert ctx.memory()[0] == used_before  # nothing allocated through the context
        assert torch.equal(d, d_ref)
        assert torch.equal(s, s_ref)
        assert st["d_max_gy"] == ref["d_max_gy"]
        assert st["s_thr"] == pytest.approx(ref["s_thr"], rel=1e-12)
        for k in ("e_deposited", "e_incident", "e_escaped", "e_rest", "histories", "n_batches"):
            assert st[k] == ref[k], k
        if call == 0:
            # more histories between the two calls: the array keeps nothing stale
            ctx.run([plan], [9_995])
            ref = ctx.plan_result(plan, 0.5, d_ref.data_ptr(), s_ref.data_ptr())
            assert ref["histories"] % n_batches == 0
            used_before = ctx.memory()[0]
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    ctx.close()


def test_noalloc_rejects_bad_arguments():
    import torch
    ctx = make_ctx()
    ph = W.homogeneous((8, 8, 8), 1.0, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, W.pencil(W.PHOTON, 1.0, 4.0, 4.0), 1, 8)
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    assert _noalloc(ctx, plan, d, d)[0] == g.ERR_STATE  # no histories yet
    ctx.run([plan], [1000])
    st = g.RunStats()
    L = g.lib()
    assert L.gpumcd_plan_result_noalloc(ctx.h, plan, 0.5, None, d.data_ptr(), None,
                                        ctypes.byref(st)) == g.ERR_INVALID_ARG
    assert L.gpumcd_plan_result_noalloc(ctx.h, 999, 0.5, d.data_ptr(), d.data_ptr(), None,
                                        ctypes.byref(st)) == g.ERR_NOT_FOUND
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    ctx.close()


def test_noalloc_rejects_phantoms_above_the_limit():
    import torch
    n = 407  # 407^3 = 67,419,143 > 2^26 voxels
    assert n ** 3 > 67108864
    ctx = make_ctx()
    ph = W.homogeneous((n, n, n), 0.1, W.MAT_WATER, 1.0)
    pid = ctx.create_phantom(ph)
    plan = ctx.plan_open(pid, W.pencil(W.PHOTON, 1.0, 20.0, 20.0), 1, 8)
    ctx.run([plan], [100])
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(ctx, plan, d, d)[0] == g.ERR_INVALID_ARG
    ctx.plan_close(plan)
    ctx.destroy_phantom(pid)
    ctx.close()

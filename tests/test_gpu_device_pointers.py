"""The device-pointer forms of the C ABI (PyTorch tensors passed zero-copy, the
work enqueued on the caller's stream) give the results of the host forms bit
for bit: a phantom made from device arrays and a dose returned into device
arrays."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import ledger_exact, make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("particle", [W.ELECTRON, W.PHOTON])
def test_device_pointer_calls_equal_host_calls(particle):
    import torch

    ctx = make_ctx()
    ph = W.z_slabs((20, 18, 24), 0.5, [(3.0, W.MAT_WATER, 1.0), (2.0, W.MAT_BONE, 1.85),
                                        (4.0, W.MAT_LUNG, 0.26), (1e9, W.MAT_WATER, 1.0)])
    src = W.Source(particle, W.BEAM_SQUARE, energy=9.0, center_cm=(5.0, 4.5), field_cm=4.0)
    host_pid = ctx.create_phantom(ph)
    mat = torch.from_numpy(np.ascontiguousarray(ph.mat)).cuda()
    rho = torch.from_numpy(np.ascontiguousarray(ph.rho)).cuda()
    d = torch.zeros(ph.nvox, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(d)
    torch.cuda.synchronize()  # the tensors are ready before another stream reads them
    stream = torch.cuda.Stream()
    dev_pid = ctx.create_phantom_device(ph.dims, ph.voxel_cm, mat.data_ptr(), rho.data_ptr(),
                                        stream.cuda_stream)
    st = ctx.simulate_device(dev_pid, src, 30_000, 5, d.data_ptr(), s.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    r = ctx.simulate(host_pid, src, 30_000, 5, nvox=ph.nvox)
    assert np.array_equal(r.dose, d.cpu().numpy()) and np.array_equal(r.sigma, s.cpu().numpy())
    for k in ("histories", "e_incident", "e_deposited", "e_escaped", "e_rest"):
        assert r.stats[k] == st[k], k
    assert ledger_exact(st) and st["e_deposited"] > 0
    ctx.destroy_phantom(host_pid)
    ctx.destroy_phantom(dev_pid)
    ctx.close()

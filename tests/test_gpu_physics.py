"""GPU tables, RNG and samplers against the oracle and the physics (CUDA path
through the C ABI)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._stats import chi2_pvalue, within_sigma
from tests.gpu_common import make_ctx

pytestmark = pytest.mark.gpu
G = 512
MC2 = 0.51099895


@pytest.fixture(scope="module")
def ctx():
    c = make_ctx()
    yield c
    c.close()


def test_tables_match_oracle_closed_forms(ctx):
    """Each FP32 table entry is the oracle's FP64 closed form at that grid
    energy, rounded (the grid energy itself is returned as FP32)."""
    grids = ctx.get_tables(3).astype(np.float64)
    ph = ctx.get_tables(0).reshape(4, 3, G)
    el = ctx.get_tables(1).reshape(4, 4, G)
    P = W.DEFAULT_PHYSICS
    for m, mat in enumerate(W.MATERIALS):
        for i in range(0, G, 7):
            E = grids[i]
            mt = oracle.xs("mu_total", mat, E)
            assert ph[m, 0, i] == pytest.approx(mt, rel=3e-6)
            assert ph[m, 1, i] == pytest.approx(oracle.xs("mu_compton", mat, E), rel=3e-6)
            assert ph[m, 2, i] == pytest.approx(oracle.xs("mu_photo", mat, E), rel=5e-6)
            T = grids[G + i]
            L = oracle.xs("l_col", mat, T, P.t_c) + oracle.xs("l_rad", mat, T, P.k_c)
            sm = oracle.xs("sigma_moller", mat, T, P.t_c)
            sb = oracle.xs("sigma_brem", mat, T, P.k_c)
            assert el[m, 0, i] == pytest.approx(L, rel=3e-6)
            assert el[m, 1, i] == pytest.approx(sm + sb, rel=3e-6, abs=1e-6)
            assert el[m, 2, i] == pytest.approx(sb, rel=3e-6, abs=1e-6)
            assert el[m, 3, i] == pytest.approx(oracle.xs("ms_lambda1_inv", mat, T), rel=5e-6)
    lna = ctx.get_tables(2).astype(np.float64)
    L = oracle.lib()
    lg = np.linspace(math.log(1e-8), math.log(20.0), 512)
    for i in range(0, 512, 9):
        assert lna[i] == pytest.approx(math.log(L.om_ms_solve_a(math.exp(lg[i]))), abs=2e-5)


def test_philox_matches_curand_and_oracle(ctx):
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8] = 0
    ctr[8:16] = 0xFFFFFFFF
    # cuRAND reaches counter word y through its 64-bit offset 4 (y:x): keep
    # 4 (y:x) below 2^64 (the generator itself is the same for every counter)
    ctr[:, 1] &= 0x3FFFFFFF
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0x12345678, 0x9ABCDEF0]):
        ours = ctx.debug_philox(ctr, key)
        ref = ctx.debug_philox(ctr, key, use_curand=True)
        assert np.array_equal(ours, ref)
        for i in range(0, 4096, 97):
            o = oracle.philox([int(v) for v in ctr[i]], key)
            assert np.array_equal(o.astype(np.uint32), ours[i])


def _kn(k):
    def f(c):
        r = 1.0 / (1.0 + k * (1.0 - c))
        return r * r * (r + 1.0 / r - (1.0 - c * c))
    return f


@pytest.mark.parametrize("E", [0.05, 0.511, 5.0, 15.0])
def test_kn_sampler(ctx, E):
    c = ctx.debug_sample(0, E, 400_000, 3).astype(np.float64)
    grid = np.concatenate([1.0 - np.geomspace(2.0, 1e-6, 20001), [1.0]])
    assert chi2_pvalue(c, _kn(E / MC2), grid) > 0.01


@pytest.mark.parametrize("T", [0.3, 2.0, 10.0])
def test_sauter_sampler(ctx, T):
    g = T / MC2 + 1
    beta = math.sqrt(1 - 1 / g ** 2)
    f = lambda c: (1 - c * c) / (1 - beta * c) ** 4 * (1 + 0.5 * g * (g - 1) * (g - 2) * (1 - beta * c))  # noqa
    c = ctx.debug_sample(1, T, 400_000, 4).astype(np.float64)
    grid = np.concatenate([[-1.0], 1.0 - np.geomspace(2.0, 1e-7, 30000)[1:], [1.0]])
    assert chi2_pvalue(c, f, grid) > 0.01


@pytest.mark.parametrize("T", [0.6, 3.0, 15.0])
def test_moller_sampler(ctx, T):
    L = oracle.lib()
    e = ctx.debug_sample(2, T, 400_000, 5).astype(np.float64)
    assert e.min() >= 0.2 / T * (1 - 1e-6) and e.max() <= 0.5 + 1e-6
    grid = np.geomspace(0.2 / T, 0.5, 20001)
    assert chi2_pvalue(e, lambda x: L.om_moller_dsigma_deps(T, x), grid) > 0.01


@pytest.mark.parametrize("T", [1.0, 15.0])
def test_brem_sampler(ctx, T):
    L = oracle.lib()
    m = oracle.material(W.BONE)
    k = ctx.debug_sample(3, T, 400_000, 6, material=W.MAT_BONE).astype(np.float64)
    grid = np.geomspace(0.01, T, 20001)
    assert chi2_pvalue(k, lambda x: L.om_brem_dsigma_dk(m, T, x), grid) > 0.01


@pytest.mark.parametrize("g1", [1e-4, 0.05, 0.7, 5.0])
def test_ms_sampler_mean(ctx, g1):
    mu = ctx.debug_sample(4, g1, 1_000_000, 7).astype(np.float64)
    m1 = 2 * mu.mean()
    s = 2 * mu.std() / math.sqrt(len(mu))
    # the ln(a) table is interpolated: allow 1e-3 relative on top of 3 sigma
    assert abs(m1 - (-math.expm1(-g1))) <= 3 * s + 1e-3 * (-math.expm1(-g1))


def test_spectrum_sampler(ctx):
    from scipy import stats
    pl = W.config3(n=16, voxel_cm=1.0)
    e = ctx.debug_sample(5, 0.0, 1_000_000, 8, src=pl.source).astype(np.float64)
    edges, w = pl.source.spectrum_edges, pl.source.spectrum_weights
    counts, _ = np.histogram(e, bins=edges)
    assert stats.chisquare(counts, w * len(e) / w.sum()).pvalue > 0.001

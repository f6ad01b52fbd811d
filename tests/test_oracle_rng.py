"""Quality checks of the oracle's Philox4x32-10.

The oracle only needs a good generator to be a correct Monte Carlo; these CPU
checks cover uniformity, bit balance, counter and key sensitivity.  Its exact
identity with the published Philox4x32-10 is pinned on the GPU against cuRAND's
Philox4_32_10 device generator
(tests/test_gpu_physics.py::test_philox_matches_curand_and_oracle).
"""
import numpy as np
from scipy import stats

import oracle


def _block(n, key=(7, 11), lane=(0, 0, 0)):
    out = np.empty((n, 4), dtype=np.uint64)
    for i in range(n):
        out[i] = oracle.philox((i, lane[0], lane[1], lane[2]), key)
    return out


def test_uniform_words():
    w = _block(20000).ravel().astype(np.float64) / 2.0 ** 32
    assert stats.kstest(w, "uniform").pvalue > 0.01
    counts, _ = np.histogram(w, bins=64, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 0.01


def test_bit_balance_and_serial_correlation():
    w = _block(20000).ravel()
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    frac = bits.mean(axis=0)
    n = len(w)
    assert np.all(np.abs(frac - 0.5) < 4 * 0.5 / np.sqrt(n))
    u = w.astype(np.float64) / 2.0 ** 32
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 4 / np.sqrt(n)


def test_avalanche_on_counter_and_key():
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(300):
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        a = oracle.philox(ctr, key)
        word, bit = int(rng.integers(0, 6)), int(rng.integers(0, 32))
        if word < 4:
            ctr[word] ^= 1 << bit
        else:
            key[word - 4] ^= 1 << bit
        b = oracle.philox(ctr, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    flips = np.array(flips)
    assert abs(flips.mean() - 64.0) < 1.5
    assert flips.min() > 30


def test_distinct_counters_give_distinct_blocks():
    b = _block(5000)
    keys = {tuple(r) for r in b.tolist()}
    assert len(keys) == 5000

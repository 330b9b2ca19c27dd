"""The seeded input generators (no shortest-path arithmetic): SplitMix64
against its published first outputs, and the batch workload's parameters --
n log-uniform in [2^10, 2^18) and the average degree uniform in [4, 32] --
against the same draws evaluated in exact Python arithmetic."""
import math

import numpy as np

import graphgen as gg


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 started at state 0 (Steele, Lea & Flood 2014)
    assert gg.splitmix64_nth(0, 0) == 0xE220A8397B1DCDAF
    assert gg.splitmix64_nth(0, 1) == 0x6E789E6AA1B965F4
    assert gg.splitmix64_nth(0, 2) == 0x06C45D188009454F


def test_batch_params_follow_their_definition():
    seed, count = 12345, 4000
    n, m, seeds, _ = gg.batch_params(count, 10, 18, 4, 32, 0, seed)
    checked = 0
    for g in range(count):
        u = gg.splitmix64_nth(seed, 2 * g) >> 32
        v = gg.splitmix64_nth(seed, 2 * g + 1) >> 32
        x = 2.0 ** (10 + 8 * u / 2**32)
        if abs(x - round(x)) > 1e-6:  # skip draws within rounding distance of an integer
            assert int(n[g]) == math.floor(x), (g, x, n[g])
            checked += 1
        assert int(m[g]) == (int(n[g]) * ((4 << 32) + 28 * v) + (1 << 31)) >> 32
        assert int(seeds[g]) == seed + ((g + 1) << 20)
    assert checked > 0.99 * count


def test_batch_params_are_log_uniform():
    n, m, _, _ = gg.batch_params(40000, 10, 18, 4, 32, 1, 777)
    assert n.min() >= 1 << 10 and n.max() < 1 << 18
    h = np.histogram(np.log2(n.astype(np.float64)), bins=16, range=(10, 18))[0]
    expect = 40000 / 16
    chi2 = float(((h - expect) ** 2 / expect).sum())
    assert chi2 < 40.0, h  # 15 degrees of freedom: far above the 99.9 % point is a broken draw
    d = m / n
    assert d.min() >= 4.0 - 1e-3 and d.max() <= 32.0 + 1e-3
    hd = np.histogram(d, bins=7, range=(4, 32))[0]
    assert (abs(hd - 40000 / 7) < 5 * math.sqrt(40000 / 7)).all(), hd

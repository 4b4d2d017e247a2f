"""Pins of the counter-based normal generator (SplitMix64 + Box-Muller)."""
import math

import numpy as np
from scipy import stats


def test_splitmix64_is_a_bijection_on_a_sample(orc):
    xs = [orc.splitmix64(z) for z in range(20000)]
    assert len(set(xs)) == len(xs)


def test_splitmix64_matches_a_python_restatement(orc):
    M = (1 << 64) - 1

    def sm(z):
        z = (z + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    for z in [0, 1, 2, 12345, M, 1 << 63]:
        assert orc.splitmix64(z) == sm(z)


def test_box_muller_restatement(orc):
    M = (1 << 64) - 1
    seed = 987654321
    for i in [0, 1, 17, 10**9 + 7]:
        a = orc.splitmix64(seed ^ (2 * i))
        b = orc.splitmix64(seed ^ (2 * i + 1))
        u1 = ((a >> 11) + 1) / 2.0 ** 53
        u2 = ((b >> 11) + 1) / 2.0 ** 53
        ref = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
        assert abs(orc.rng_normal(seed, i, 1)[0] - ref) < 1e-15
        assert b <= M


def test_normal_distribution(orc):
    x = orc.rng_normal(42, 0, 200000)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1) < 0.01
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # counter based: any window is reproducible independently
    assert np.array_equal(orc.rng_normal(42, 1000, 10), x[1000:1010])
    assert not np.array_equal(orc.rng_normal(43, 0, 10), x[:10])

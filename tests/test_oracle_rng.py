"""Pins of the counter-based normal generator (SplitMix64 + Box-Muller)."""
import math

import numpy as np
from scipy import stats

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_splitmix64_reproduces_the_published_stream(orc):
    # The first five outputs of SplitMix64 seeded with 1234567, as published
    # with the generator's reference implementation (splitmix64.c, Vigna) and
    # used as its test vector.  Output n (1-based) of the stream from state x0
    # is xo_splitmix64(x0 + (n - 1) gamma).
    published = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                 4593380528125082431, 16408922859458223821]
    got = [orc.splitmix64((1234567 + n * GAMMA) & M64) for n in range(5)]
    assert got == published


def test_splitmix64_is_a_bijection_on_a_sample(orc):
    xs = [orc.splitmix64(z) for z in range(20000)]
    assert len(set(xs)) == len(xs)


def test_box_muller_on_the_stream_outputs(orc):
    # entry i takes outputs 2i+1 and 2i+2 of the stream whose state is
    # k = splitmix64(seed); Box-Muller: sqrt(-2 ln u1) cos(2 pi u2)
    seed = 987654321
    k = orc.splitmix64(seed)
    for i in [0, 1, 17, 10**9 + 7]:
        a = orc.splitmix64((k + 2 * i * GAMMA) & M64)
        b = orc.splitmix64((k + (2 * i + 1) * GAMMA) & M64)
        u1 = ((a >> 11) + 1) / 2.0 ** 53
        u2 = ((b >> 11) + 1) / 2.0 ** 53
        assert 0.0 < u1 <= 1.0 and 0.0 < u2 <= 1.0
        ref = math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)
        assert abs(orc.rng_normal(seed, i, 1)[0] - ref) < 1e-15


def test_normal_distribution(orc):
    x = orc.rng_normal(42, 0, 200000)
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1) < 0.01
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # counter based: any window is reproducible independently
    assert np.array_equal(orc.rng_normal(42, 1000, 10), x[1000:1010])
    assert not np.array_equal(orc.rng_normal(43, 0, 10), x[:10])


def test_nearby_seeds_give_independent_vectors(orc):
    # Seeds seed, seed + 1, ... (the starts of the finite-temperature Lanczos
    # runs) and seeds differing in single bits must not give permutations or
    # shifts of one vector: the sorted values differ and the pairwise
    # correlations, also against shifted copies, are of order 1/sqrt(n).
    n = 4096
    seeds = [1, 2, 3, 4, 5, 17, 1 ^ (1 << 40), 1000]
    vs = [orc.rng_normal(s, 0, n) for s in seeds]
    for a in range(len(vs)):
        for b in range(a + 1, len(vs)):
            assert not np.allclose(np.sort(vs[a]), np.sort(vs[b]))
            for shift in (0, 1, 2):
                c = np.corrcoef(vs[a][shift:], vs[b][:n - shift])[0, 1]
                assert abs(c) < 5.0 / math.sqrt(n)

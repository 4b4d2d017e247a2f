"""Pins of the oracle's U(1) basis and index maps (Sec. 3.1, Sec. 5.2)."""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("N", range(1, 15))
def test_enumeration_brute_force(orc, N):
    for nup in range(N + 1):
        st = orc.enumerate_states(N, nup)
        brute = [w for w in range(2 ** N) if bin(w).count("1") == nup]
        assert st.tolist() == brute
        assert st.size == math.comb(N, nup) == orc.binom(N, nup)


@pytest.mark.parametrize("N", [1, 5, 12, 16, 20])
def test_sector_dims_sum_to_full_space(orc, N):
    assert sum(orc.binom(N, k) for k in range(N + 1)) == 2 ** N


def test_binomials_of_the_workloads(orc):
    # Block sizes of the chain N=16, ladder N=28, 4x8 N=32 and 6x6 N=36 at Sz=0.
    assert orc.binom(16, 8) == 12870
    assert orc.binom(28, 14) == 40116600
    assert orc.binom(32, 16) == 601080390
    assert orc.binom(36, 18) == 9075135300
    for n in range(0, 65):
        for k in (0, n // 3, n // 2, n):
            assert orc.binom(n, k) == math.comb(n, k)


@pytest.mark.parametrize("N,nup", [(4, 2), (10, 3), (12, 6), (16, 8), (16, 5)])
def test_counting_index_equals_search(orc, N, nup):
    st = orc.enumerate_states(N, nup)
    for k, s in enumerate(st):
        s = int(s)
        assert orc.index_search(st, s) == k
        assert orc.index_count(N, nup, s) == k
        assert orc.state_count(N, nup, k) == s


def test_index_of_absent_state(orc):
    st = orc.enumerate_states(8, 4)
    assert orc.index_search(st, 0b111) == -1
    assert orc.index_count(8, 4, 0b111) == -1
    assert orc.index_count(8, 4, 0b1111 << 8) == -1  # beyond N bits


def test_counting_index_at_n36(orc):
    rng = np.random.default_rng(0)
    N, nup = 36, 18
    assert orc.index_count(N, nup, (1 << 18) - 1) == 0
    assert orc.index_count(N, nup, ((1 << 18) - 1) << 18) == math.comb(36, 18) - 1
    for _ in range(200):
        k = int(rng.integers(0, math.comb(36, 18)))
        s = orc.state_count(N, nup, k)
        assert bin(s).count("1") == nup and s < (1 << N)
        assert orc.index_count(N, nup, s) == k

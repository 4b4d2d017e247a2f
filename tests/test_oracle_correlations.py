"""Pins of the oracle's two-point spin correlations (Sec. 3.7 inner with the
SzSz and SdotS operators on arbitrary site pairs)."""
import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W


def _ground_state(orc, N, nup, bonds, J):
    st = orc.enumerate_states(N, nup)
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    return st, w, V


def test_two_site_singlet(orc):
    """N=2, one bond: the singlet (|01> - |10>)/sqrt(2) has <S0.S1> = -3/4,
    <Sz0 Sz1> = -1/4; the Sz=0 triplet has +1/4 and -1/4."""
    st = orc.enumerate_states(2, 1)  # [0b01, 0b10]
    singlet = np.array([1.0, -1.0]) / np.sqrt(2)
    triplet = np.array([1.0, 1.0]) / np.sqrt(2)
    pairs = [(0, 1), (1, 0), (0, 0)]
    assert np.allclose(orc.correlations(2, st, pairs, "ss", singlet), [-0.75, -0.75, 0.75], atol=1e-15)
    assert np.allclose(orc.correlations(2, st, pairs, "zz", singlet), [-0.25, -0.25, 0.25], atol=1e-15)
    assert np.allclose(orc.correlations(2, st, pairs, "ss", triplet), [0.25, 0.25, 0.75], atol=1e-15)


@pytest.mark.parametrize("N", [8, 10, 12])
def test_singlet_ground_state_rules(orc, N):
    """Chain ground state (a singlet, Lieb-Mattis): <Si.Sj> = 3 <Szi Szj>;
    sum_j <S0.Sj> = <S0.S_tot> = 0; sum_{i<j} <Si.Sj> = (S^2 - 3N/4)/2 = -3N/8;
    the nearest-neighbour value is E0/N; <Szi Szi> = 1/4."""
    bonds = W.chain(N)
    st, w, V = _ground_state(orc, N, N // 2, bonds, np.ones(N))
    psi = V[:, 0]
    pairs = [(0, j) for j in range(N)]
    ss = orc.correlations(N, st, pairs, "ss", psi)
    zz = orc.correlations(N, st, pairs, "zz", psi)
    assert np.abs(ss - 3 * zz).max() < 1e-12
    assert abs(ss.sum()) < 1e-12
    assert abs(zz[0] - 0.25) < 1e-15 and abs(ss[0] - 0.75) < 1e-15
    allp = [(i, j) for i in range(N) for j in range(i + 1, N)]
    assert abs(orc.correlations(N, st, allp, "ss", psi).sum() + 3 * N / 8) < 1e-11
    assert abs(ss[1] - w[0] / N) < 1e-12
    # antiferromagnetic signs alternate
    assert np.all(np.sign(zz[1:]) == np.array([(-1) ** j for j in range(1, N)]))


def test_sz_sum_rule_any_state(orc):
    """In the Sz = 0 block sum_j Sz_j = 0, so sum_j <psi|Sz_0 Sz_j|psi> = 0
    for every state, not only eigenstates."""
    N = 10
    st = orc.enumerate_states(N, 5)
    psi = orc.rng_normal(3, 0, st.size)
    zz = orc.correlations(N, st, [(0, j) for j in range(N)], "zz", psi)
    assert abs(zz.sum()) < 1e-12 * np.dot(psi, psi)


def test_ss_is_the_bond_form(orc):
    """<psi|S_i.S_j|psi> equals the bilinear form of the bond (i, j) at g = x."""
    N = 11
    st = orc.enumerate_states(N, 4)
    pairs = W.random_bonds(N, 15, 2)
    psi = orc.rng_normal(5, 0, st.size)
    assert np.abs(orc.correlations(N, st, pairs, "ss", psi) - orc.bond_forms(N, st, pairs, psi, psi)).max() < 1e-12

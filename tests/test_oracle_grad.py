"""Pins of the per-bond bilinear forms and of dE0/dJ (Sec. 3.7 inner)."""
import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W


def _ground(orc, N, st, bonds, J):
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    return w, V[:, 0]


def test_bond_forms_are_the_coupling_derivative(orc):
    N, nup = 10, 5
    bonds = W.random_bonds(N, 18, 3)
    J = W.uniform_couplings(18, 4)
    st = orc.enumerate_states(N, nup)
    rng = np.random.default_rng(5)
    g, x = rng.standard_normal((2, st.size))
    dJ = orc.bond_forms(N, st, bonds, g, x)
    # <g|H(J)|x> is linear in J: central differences are exact up to rounding
    for b in range(18):
        e = np.zeros(18); e[b] = 0.5
        f = lambda JJ: g @ orc.apply_u1(N, st, bonds, JJ, x)  # noqa: E731
        assert abs((f(J + e) - f(J - e)) / 1.0 - dJ[b]) < 1e-10 * (1 + abs(dJ[b]))
    assert abs(J @ dJ - g @ orc.apply_u1(N, st, bonds, J, x)) < 1e-10 * np.abs(g @ x + 1)


def test_hellmann_feynman_ladder(orc):
    """C3 pattern at small size: a 5-rung periodic ladder, each rung twice."""
    L = 5
    bonds = W.ladder(L, 2)
    N = 2 * L
    J = W.uniform_couplings(bonds.shape[0], 3)
    st = orc.enumerate_states(N, L)
    w, psi = _ground(orc, N, st, bonds, J)
    assert w[1] - w[0] > 1e-3  # unique singlet ground state
    hf = orc.bond_forms(N, st, bonds, psi, psi)
    h = 1e-5
    for b in range(bonds.shape[0]):
        e = np.zeros_like(J); e[b] = h
        fd = (_ground(orc, N, st, bonds, J + e)[0][0] - _ground(orc, N, st, bonds, J - e)[0][0]) / (2 * h)
        assert abs(fd - hf[b]) < 1e-7
    assert abs(J @ hf - w[0]) < 1e-12             # Euler: H is degree-1 in J
    rung_a, rung_b = hf[2 * L:3 * L], hf[3 * L:]
    assert np.abs(rung_a - rung_b).max() < 1e-12  # two copies of each rung
    assert np.all(hf <= 0.25 + 1e-12) and np.all(hf >= -0.75 - 1e-12)


def test_singlet_correlator_isotropy(orc):
    N = 8
    bonds, J = W.chain(N), np.ones(N)
    st = orc.enumerate_states(N, 4)
    _, psi = _ground(orc, N, st, bonds, J)
    hf = orc.bond_forms(N, st, bonds, psi, psi)
    # <Sz_i Sz_j> from the diagonal only; singlet: <S_i.S_j> = 3 <Sz_i Sz_j>
    for b, (i, j) in enumerate(bonds):
        zz = sum(p * p * (0.25 if ((int(s) >> i) & 1) == ((int(s) >> j) & 1) else -0.25)
                 for s, p in zip(st, psi))
        assert abs(hf[b] - 3 * zz) < 1e-12


@pytest.mark.parametrize("N", [8, 12])
def test_lanczos_matches_dense(orc, N):
    bonds = W.random_bonds(N, 2 * N, N)
    J = W.uniform_couplings(2 * N, N)
    st = orc.enumerate_states(N, N // 2)
    w, psi = _ground(orc, N, st, bonds, J)
    mv = lambda v: orc.apply_u1(N, st, bonds, J, v)  # noqa: E731
    v0 = orc.rng_normal(9, 0, st.size)
    a, b = orc.lanczos(mv, st.size, v0, min(st.size, 120))
    assert abs(orc.tridiag_eigvals(a, b)[0] - w[0]) < 1e-10 * abs(w[0])
    e0, phi = orc.lanczos_ground_state(mv, st.size, v0, min(st.size, 120))
    assert abs(e0 - w[0]) < 1e-10 * abs(w[0])
    assert np.linalg.norm(mv(phi) - e0 * phi) < 1e-6

"""Pins of the oracle's time evolution exp(-z H) psi0 (Sec. 3.6.2)."""
import numpy as np

from paper_2505_02901_gb300 import workloads as W


def test_two_site_closed_form(orc):
    """H = J S0.S1 on the Sz=0 pair: |01> = (|T0> + |S>)/sqrt(2) with E_T =
    J/4 and E_S = -3J/4, so <01|e^{-iHt}|01> = (e^{-iJt/4} + e^{3iJt/4})/2 and
    |<01|psi(t)>|^2 = cos^2(J t / 2)."""
    st = orc.enumerate_states(2, 1)  # [0b01, 0b10]
    J = 1.3
    H = orc.dense_u1(2, st, W.chain(2), [J])
    for t in (0.0, 0.4, 1.7, 5.0):
        psi = orc.evolve_dense(H, np.array([1.0, 0.0]), 1j * t)
        assert abs(psi[0] - (np.exp(-1j * J * t / 4) + np.exp(3j * J * t / 4)) / 2) < 1e-14
        assert abs(abs(psi[0]) ** 2 - np.cos(J * t / 2) ** 2) < 1e-14


def test_unitarity_group_property_and_energy(orc):
    N = 10
    st = orc.enumerate_states(N, 5)
    bonds, J = W.random_bonds(N, 2 * N, 1), W.uniform_couplings(2 * N, 1)
    H = orc.dense_u1(N, st, bonds, J)
    psi0 = orc.rng_normal(4, 0, st.size) + 1j * orc.rng_normal(5, 0, st.size)
    a = orc.evolve_dense(H, psi0, 0.7j)
    b = orc.evolve_dense(H, orc.evolve_dense(H, psi0, 0.3j), 0.4j)
    assert np.abs(a - b).max() < 1e-12
    assert abs(np.linalg.norm(a) - np.linalg.norm(psi0)) < 1e-12
    e = lambda v: np.vdot(v, H @ v).real / np.vdot(v, v).real  # noqa: E731
    assert abs(e(a) - e(psi0)) < 1e-12
    # backwards in time returns the start
    assert np.abs(orc.evolve_dense(H, a, -0.7j) - psi0).max() < 1e-12


def test_imaginary_time_projects_to_ground_state(orc):
    N = 12
    st = orc.enumerate_states(N, 6)
    H = orc.dense_u1(N, st, W.chain(N), np.ones(N))
    w = np.linalg.eigvalsh(H)
    psi = orc.evolve_dense(H, orc.rng_normal(2, 0, st.size), 40.0)
    e = np.vdot(psi, H @ psi).real / np.vdot(psi, psi).real
    assert abs(e - w[0]) < 1e-10

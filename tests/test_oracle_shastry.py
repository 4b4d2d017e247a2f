"""The Shastry-Sutherland model (the paper's thermodynamics example, Sec. 4):
the product of singlets on the orthogonal dimers is an exact eigenstate with
energy -3 J N / 8 for every J' (each J' triangle's two bonds to a dimer cancel
on its singlet), and in the dimer phase it is the ground state.  A dropped or
mis-signed bond term anywhere in the product breaks the cancellation."""
import math

import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W


def dimer_state(states, dimers):
    """prod_d (|up_i dn_j> - |dn_i up_j>)/sqrt 2 on the U(1) block (nup = N/2)."""
    psi = np.zeros(states.size)
    s = states.astype(np.uint64)
    ok = np.ones(states.size, dtype=bool)
    sign = np.ones(states.size)
    for i, j in dimers:
        bi = (s >> np.uint64(i)) & np.uint64(1)
        bj = (s >> np.uint64(j)) & np.uint64(1)
        ok &= bi != bj
        sign *= np.where(bi == 1, 1.0, -1.0)
    psi[ok] = sign[ok] * 2.0 ** (-len(dimers) / 2)
    return psi


def test_dimer_pattern():
    for Lx, Ly in ((4, 4), (4, 6), (6, 6)):
        bonds, J, dimers = W.shastry_sutherland(Lx, Ly)
        N = Lx * Ly
        assert sorted(dimers.reshape(-1).tolist()) == list(range(N))  # every site once
        assert len(bonds) == N // 2 + 2 * N and np.count_nonzero(J == 1.0) == N // 2
        # each dimer is a plaquette diagonal: its sites differ by one step in x and in y
        for i, j in dimers:
            dx = (j % Lx - i % Lx) % Lx
            dy = (j // Lx - i // Lx) % Ly
            assert dx in (1, Lx - 1) and dy in (1, Ly - 1)
        with pytest.raises(ValueError):
            W.shastry_sutherland(4, 5)


@pytest.mark.parametrize("Lx,Ly,Jp", [(4, 4, 0.5), (4, 4, 1.3), (4, 6, 0.5)])
def test_dimer_product_is_exact_eigenstate(orc, Lx, Ly, Jp):
    bonds, J, dimers = W.shastry_sutherland(Lx, Ly, 1.0, Jp)
    N = Lx * Ly
    st = orc.enumerate_states(N, N // 2)
    psi = dimer_state(st, dimers)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    assert np.count_nonzero(psi) == 2 ** (N // 2)
    hpsi = orc.apply_u1(N, st, bonds, J, psi)
    assert np.abs(hpsi - (-3.0 * N / 8) * psi).max() < 1e-13


def test_dimer_phase_ground_energy(orc):
    """At J'/J = 0.5 (inside the dimer phase) the 16-site cluster's ground
    energy is -3N/8 = -6, and the first excitation lies above it."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    bonds, J, _ = W.shastry_sutherland(4, 4, 1.0, 0.5)
    st = orc.enumerate_states(16, 8)
    op = LinearOperator((st.size, st.size), matvec=lambda v: orc.apply_u1(16, st, bonds, J, v))
    w = np.sort(eigsh(op, k=2, which="SA", tol=1e-12)[0])
    assert abs(w[0] + 6.0) < 1e-10
    assert w[1] > w[0] + 0.1
    assert math.isclose(-3 * 16 / 8, -6.0)

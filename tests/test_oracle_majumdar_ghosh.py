"""The J1-J2 chain at the Majumdar-Ghosh point J2 = J1/2: the two
nearest-neighbour dimer coverings D1 = s(0,1) s(2,3) ... and
D2 = s(1,2) ... s(N-1,0) (s = singlet) are exact eigenstates with energy
-3 N J1 / 8 and span the ground space.  Translation swaps them; reflection
maps D1 to (-1)^(N/2) D2, so for even N/2 the ground states are D1 + D2 in
the (k = 0, even) sector and D1 - D2 in the (k = pi, odd) sector of D_N."""
import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W
from tests.test_oracle_shastry import dimer_state


def coverings(N):
    return ([(2 * j, 2 * j + 1) for j in range(N // 2)],
            [(2 * j + 1, (2 * j + 2) % N) for j in range(N // 2)])


@pytest.mark.parametrize("N", [8, 12, 16])
def test_dimer_coverings_are_ground_states(orc, N):
    from scipy.sparse.linalg import LinearOperator, eigsh
    bonds, J = W.chain_j1j2(N)
    st = orc.enumerate_states(N, N // 2)
    for cov in coverings(N):
        d = dimer_state(st, cov)
        assert np.abs(orc.apply_u1(N, st, bonds, J, d) + 3 * N / 8 * d).max() < 1e-13
    op = LinearOperator((st.size,) * 2, matvec=lambda v: orc.apply_u1(N, st, bonds, J, v))
    w = np.sort(eigsh(op, k=3, which="SA", tol=1e-12)[0])
    assert np.abs(w[:2] + 3 * N / 8).max() < 1e-10
    assert w[2] > -3 * N / 8 + 0.2


@pytest.mark.parametrize("N", [8, 12])
def test_dihedral_sectors_of_the_ground_states(orc, N):
    bonds, J = W.chain_j1j2(N)
    low = {}
    for m in (0, N // 2):
        for parity in (1, -1):
            blk = orc.SymBlock(N, N // 2, W.chain_dihedral(N), W.chain_dihedral_characters(N, m, parity))
            low[(m, parity)] = np.linalg.eigvalsh(blk.dense(bonds, J))[0].real
    assert abs(low[(0, 1)] + 3 * N / 8) < 1e-12 and abs(low[(N // 2, -1)] + 3 * N / 8) < 1e-12
    assert low[(0, -1)] > -3 * N / 8 + 0.2 and low[(N // 2, 1)] > -3 * N / 8 + 0.2

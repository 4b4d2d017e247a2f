"""The J1-J2 chain at the Majumdar-Ghosh point on the GPU: the dimer
coverings are exact eigenstates of the U(1) product with energy -3N/8, and
the D_N blocks (ring search of the orbit) hold that energy exactly in the
(k = 0, even) and (k = pi, odd) sectors, the other two lying above it."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api
from tests.test_oracle_majumdar_ghosh import coverings
from tests.test_oracle_shastry import dimer_state

pytestmark = pytest.mark.gpu


def check_mg(A, orc, N):
    bonds, J = W.chain_j1j2(N)
    e = -3.0 * N / 8
    ham = A.Hamiltonian(A.Basis(N, N // 2, bonds), J)
    st = orc.enumerate_states(N, N // 2)
    for cov in coverings(N):
        d = dimer_state(st, cov)
        y = ham.apply(torch.from_numpy(d).cuda()).cpu().numpy()
        assert np.abs(y - e * d).max() < 1e-13
    low = {}
    for m in (0, N // 2):
        for parity in (1, -1):
            sym = (W.chain_dihedral(N), W.chain_dihedral_characters(N, m, parity))
            hs = A.Hamiltonian(A.Basis(N, N // 2, bonds, symmetry=sym), J)
            low[(m, parity)] = hs.lanczos(max_iter=150, seed=2)["evals"][0]
    assert abs(low[(0, 1)] - e) < 1e-9 and abs(low[(N // 2, -1)] - e) < 1e-9
    assert low[(0, -1)] > e + 0.1 and low[(N // 2, 1)] > e + 0.1


def test_majumdar_ghosh_chain24(orc):
    check_mg(api(), orc, 24)

"""Finite-temperature Lanczos on the GPU against the oracle."""
import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,R,M", [(12, 16, 20), (14, 11, 25)])
def test_ftlm_tridiagonals_match_oracle(orc, N, R, M):
    A = api()
    bonds, J = W.random_bonds(N, 2 * N, 4), W.uniform_couplings(2 * N, 4)
    st = orc.enumerate_states(N, N // 2)
    ham = A.Hamiltonian(A.Basis(N, N // 2, bonds), J)
    seed = 77
    a, b, n = ham.ftlm(R, M, seed)
    H = orc.dense_u1(N, st, bonds, J)
    tri = orc.ftlm_tridiagonals(lambda v: H @ v, [orc.rng_normal(seed + r, 0, st.size) for r in range(R)], M)
    for r, (ao, bo, _) in enumerate(tri):
        assert n[r] == M
        assert np.abs(a[r] - ao).max() <= 1e-9 * np.abs(ao).max()
        assert np.abs(b[r] - bo).max() <= 1e-9 * np.abs(bo).max()
    temps = [0.2, 1.0, 5.0]
    Z, E, C = A.ftlm_thermo(a, b, n, st.size, temps)
    ref = orc.ftlm_thermo([(a[r], b[r], 1.0) for r in range(R)], st.size, temps)
    for q, (z0, e0, c0) in enumerate(ref):
        assert abs(Z[q] / z0 - 1) < 1e-10 and abs(E[q] - e0) < 1e-10 and abs(C[q] - c0) < 1e-9


def test_ftlm_low_temperature_is_the_ground_state(orc):
    A = api()
    N = 16
    ham = A.Hamiltonian(A.Basis(N, N // 2, W.chain(N)), np.ones(N))
    e0 = ham.lanczos(max_iter=200, seed=1)["evals"][0]
    a, b, n = ham.ftlm(8, 90, 5)
    Z, E, C = A.ftlm_thermo(a, b, n, ham.dim, [0.01, 100.0])
    assert abs(E[0] - e0) < 1e-6
    # T -> infinity: E -> Tr H / dim; for the chain at Sz = 0 that is
    # N * (1/4) (1 - 2 P_anti), P_anti = 2 nup (N - nup) / (N (N - 1))
    p_anti = 2 * (N // 2) * (N - N // 2) / (N * (N - 1))
    assert abs(E[1] - N * 0.25 * (1 - 2 * p_anti)) < 0.05 * N * 0.25

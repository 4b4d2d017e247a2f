"""The Shastry-Sutherland model on the GPU (the paper's thermodynamics
example, Sec. 4) against its closed forms: the dimer-singlet product is an
exact eigenstate with energy -3 J N / 8 for any J'; in the dimer phase it is
the unique ground state, so <S_i.S_j> is -3/4 on every dimer bond and 0 on
every J' bond, and the thermal energy tends to -3 J N / 8 as T -> 0."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api
from tests.test_oracle_shastry import dimer_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("Jp", [0.5, 1.3])
def test_dimer_product_is_an_eigenstate_on_gpu(orc, Jp):
    A = api()
    bonds, J, dimers = W.shastry_sutherland(4, 6, 1.0, Jp)
    N = 24
    psi = dimer_state(orc.enumerate_states(N, N // 2), dimers)
    ham = A.Hamiltonian(A.Basis(N, N // 2, bonds), J)
    assert ham.dim == psi.size
    x = torch.from_numpy(psi).cuda()
    y = ham.apply(x).cpu().numpy()
    assert np.abs(y + 3.0 * N / 8 * psi).max() < 1e-13
    y32 = ham.apply(x.float()).double().cpu().numpy()
    assert np.abs(y32 + 3.0 * N / 8 * psi).max() < 1e-6


def test_dimer_phase_ground_state_gradient_and_ftlm(orc):
    A = api()
    bonds, J, dimers = W.shastry_sutherland(4, 4, 1.0, 0.5)
    N, nd = 16, 8
    ham = A.Hamiltonian(A.Basis(N, N // 2, bonds), J)
    e0, psi, _ = ham.ground_state(max_iter=150, seed=3)
    assert abs(e0 + 6.0) < 1e-10
    g = ham.energy_grad(psi)
    assert np.abs(g[:nd] + 0.75).max() < 1e-8
    assert np.abs(g[nd:]).max() < 1e-8
    a, b, n = ham.ftlm(8, 80, 9)
    Z, E, C = A.ftlm_thermo(a, b, n, ham.dim, [0.01])
    assert abs(E[0] + 6.0) < 1e-6

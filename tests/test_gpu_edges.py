"""Degenerate blocks and sizes through every entry point."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nup", [0, 6])
def test_one_state_blocks(nup):
    """nup = 0 or N: one state, H = sum J / 4 (all spins parallel)."""
    A = api()
    N = 6
    J = W.uniform_couplings(N, 1)
    ham = A.Hamiltonian(A.Basis(N, nup, W.chain(N)), J)
    assert ham.dim == 1
    e = J.sum() / 4
    x = torch.ones(1, dtype=torch.float64, device="cuda")
    assert abs(float(ham.apply(x)[0]) - e) < 1e-15
    info = ham.lanczos(max_iter=5, seed=1)
    assert info["n_iter"] == 1 and abs(info["evals"][0] - e) < 1e-15
    psi = torch.ones(1, dtype=torch.complex128, device="cuda")
    out, ev = ham.evolve(psi, t=2.0)
    assert abs(complex(out[0].item()) - np.exp(-2j * e)) < 1e-13
    c = ham.basis.correlations(x, [(0, 1), (2, 2)], "ss")
    assert np.allclose(c, [0.25, 0.75], atol=1e-15)
    a, b, n = ham.ftlm(3, 4, 1)
    assert np.all(n == 1) and np.allclose(a[:, 0], e, atol=1e-14)


def test_zero_pairs_and_single_step():
    A = api()
    ham = A.Hamiltonian(A.Basis(8, 4, W.chain(8)), np.ones(8))
    x = A.random_vector(ham.dim, 1, torch.float64)
    assert ham.basis.correlations(x, np.zeros((0, 2), dtype=np.int32)).size == 0
    a, b, n = ham.ftlm(8, 1, 2)
    assert np.all(n == 1)
    out, info = ham.evolve(x.to(torch.complex128), t=0.0)
    assert torch.allclose(out, x.to(torch.complex128), atol=1e-14)

"""Time evolution exp(-z H) psi0 (Sec. 3.6.2) on the GPU against the oracle."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def _cplx(orc, seed, n):
    return orc.rng_normal(seed, 0, n) + 1j * orc.rng_normal(seed + 1, 0, n)


@pytest.mark.parametrize("t,tau", [(0.5, 0.0), (2.0, 0.0), (0.0, 1.0), (1.5, 0.3)])
def test_u1_evolution_matches_oracle(orc, t, tau):
    A = api()
    N, nup = 12, 6
    bonds, J = W.random_bonds(N, 2 * N, 3), W.uniform_couplings(2 * N, 3)
    st = orc.enumerate_states(N, nup)
    H = orc.dense_u1(N, st, bonds, J)
    psi0 = _cplx(orc, 7, st.size)
    ref = orc.evolve_dense(H, psi0, tau + 1j * t)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    out, info = ham.evolve(torch.from_numpy(psi0).cuda(), t=t, tau=tau, tol=1e-13)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-10
    assert info["err"] <= 1e-13 * np.linalg.norm(psi0) * 10


@pytest.mark.parametrize("m", [0, 1, 3])
def test_symmetric_block_evolution(orc, m):
    A = api()
    N = 12
    perms, chi = W.chain_translations(N), W.chain_characters(N, m)
    blk = orc.SymBlock(N, N // 2, perms, chi)
    Hk = blk.dense(W.chain(N), np.ones(N))
    psi0 = _cplx(orc, 11 + m, blk.dim)
    ref = orc.evolve_dense(Hk, psi0, 0.8j)
    ham = A.Hamiltonian(A.Basis(N, N // 2, W.chain(N), symmetry=(perms, chi)), np.ones(N))
    out, info = ham.evolve(torch.from_numpy(psi0).cuda(), t=0.8, tol=1e-13)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-10


def test_two_site_closed_form():
    """H = J S0.S1: |<01|psi(t)>|^2 = cos^2(J t / 2) from psi0 = |01>."""
    A = api()
    J = 1.3
    ham = A.Hamiltonian(A.Basis(2, 1, W.chain(2)), [J])
    psi0 = torch.tensor([1.0 + 0j, 0.0], dtype=torch.complex128, device="cuda")
    for t in (0.4, 1.7, 5.0):
        out, info = ham.evolve(psi0, t=t)
        assert abs(abs(out[0].item()) ** 2 - np.cos(J * t / 2) ** 2) < 1e-13


def test_unitarity_energy_and_group_property(orc):
    """N=20 chain (dim 184756): the norm and <H> are conserved and
    e^{-iH(t1 + t2)} = e^{-iH t2} e^{-iH t1}."""
    A = api()
    N = 20
    ham = A.Hamiltonian(A.Basis(N, N // 2, W.chain(N)), np.ones(N))
    psi0 = torch.from_numpy(_cplx(orc, 21, ham.dim)).cuda()

    def energy(v):
        hv = ham.apply(torch.view_as_real(v).contiguous())
        return float((torch.view_as_real(v) * hv).sum() / (v.abs() ** 2).sum())

    a, ia = ham.evolve(psi0, t=1.0, tol=1e-12)
    b1, _ = ham.evolve(psi0, t=0.4, tol=1e-12)
    b, _ = ham.evolve(b1, t=0.6, tol=1e-12)
    assert abs(float(a.norm()) / float(psi0.norm()) - 1) < 1e-11
    assert abs(energy(a) - energy(psi0)) < 1e-10 * abs(energy(psi0)) + 1e-10
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 1e-10
    assert ia["n_iter"] >= 2


def test_evolve_errors():
    A = api()
    ham = A.Hamiltonian(A.Basis(6, 3, W.chain(6)), np.ones(6))
    psi = torch.zeros(ham.dim, dtype=torch.complex128, device="cuda")
    with pytest.raises(A.XDError):
        ham.evolve(psi, t=1.0, max_iter=0)
    out, info = ham.evolve(psi, t=1.0)  # exp(-zH) 0 = 0
    assert float(out.abs().max()) == 0.0 and info["n_iter"] == 0

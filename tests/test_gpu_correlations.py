"""Two-point spin correlations on the GPU against the oracle."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,nup,seed", [(12, 6, 1), (16, 8, 2), (20, 10, 3), (14, 5, 4), (24, 2, 5)])
def test_correlations_match_oracle(orc, N, nup, seed):
    A = api()
    st = orc.enumerate_states(N, nup)
    basis = A.Basis(N, nup, W.chain(N))
    pairs = [(0, j) for j in range(N)] + [(i, i) for i in range(N)]
    pairs += [tuple(p) for p in W.random_bonds(N, min(40, N * (N - 1) // 2), seed)]
    if N == 24:  # every pair, more than one launch of 256
        pairs = [(i, j) for i in range(N) for j in range(N)]
    psi = orc.rng_normal(seed, 0, st.size)
    for kind in ("ss", "zz"):
        ref = orc.correlations(N, st, pairs, kind, psi)
        got = basis.correlations(torch.from_numpy(psi).cuda(), pairs, kind)
        assert rel_l2(got, ref) <= 1e-12
        assert np.array_equal(got, basis.correlations(torch.from_numpy(psi).cuda(), pairs, kind))
        p32 = psi.astype(np.float32)
        ref32 = orc.correlations(N, st, pairs, kind, p32.astype(np.float64))
        got32 = basis.correlations(torch.from_numpy(p32).cuda(), pairs, kind)
        assert rel_l2(got32, ref32) <= 1e-12


def test_ground_state_correlations_su2(orc):
    """Chain N=18 ground state from the GPU Lanczos: a singlet, so
    <S0.Sj> = 3 <Sz0 Szj>, sum_j <S0.Sj> = 0, and <S0.S1> = E0/N."""
    A = api()
    N = 18
    ham = A.Hamiltonian(A.Basis(N, N // 2, W.chain(N)), np.ones(N))
    e0, psi, info = ham.ground_state(max_iter=200, seed=3)
    pairs = [(0, j) for j in range(N)]
    ss = ham.basis.correlations(psi, pairs, "ss")
    zz = ham.basis.correlations(psi, pairs, "zz")
    assert np.abs(ss - 3 * zz).max() < 1e-8
    assert abs(ss.sum()) < 1e-8
    assert abs(ss[1] - e0 / N) < 1e-8
    assert abs(ss[0] - 0.75) < 1e-12 and abs(zz[0] - 0.25) < 1e-12


def test_correlations_errors():
    A = api()
    basis = A.Basis(8, 4, W.chain(8))
    psi = torch.zeros(basis.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(A.XDError):
        basis.correlations(psi, [(0, 8)])
    with pytest.raises(A.XDError):
        basis.correlations(psi.to(torch.complex128), [(0, 1)])
    # symmetry-adapted blocks: pairs inside the lattice, the block's own dtype
    sym = A.Basis(8, 4, W.chain(8), symmetry=(W.chain_translations(8), W.chain_characters(8, 0)))
    zero = torch.zeros(sym.dim, dtype=torch.float64, device="cuda")
    assert np.all(sym.correlations(zero, [(0, 1), (2, 2)], "zz") == 0.0)
    with pytest.raises(A.XDError):
        sym.correlations(zero, [(0, 8)])
    with pytest.raises(A.XDError):
        sym.correlations(zero.to(torch.complex128), [(0, 1)])
    with pytest.raises(A.XDError):
        sym.correlations(zero, [(0, 1)], "xx")


"""Two-point spin correlations on symmetry-adapted blocks on the GPU: the
symmetric bond form on the orbits of the site pairs, against the oracle's
U(1) correlations of the lifted state."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api

pytestmark = pytest.mark.gpu


def _sym_case(case):
    if case == 0:  # real: D_12 on the J1-J2 chain
        b, J = W.chain_j1j2(12, 1.0, 0.3)
        return 12, 6, b, J, W.chain_dihedral(12), W.chain_dihedral_characters(12, 0, 1)
    if case == 1:  # real: the 128-element space group of the 4x4 J1-J2 lattice
        b, J = W.square_j1j2(4, 4)
        return 16, 8, b, J, W.torus_space_group(4), np.ones(128, dtype=np.complex128)
    # complex: momentum 2 pi / 12 of the chain
    return 12, 6, W.chain(12), np.ones(12), W.chain_translations(12), W.chain_characters(12, 1)


@pytest.mark.parametrize("case", range(3))
def test_symmetric_block_correlations(orc, case):
    """<psi|S_i.S_j|psi> on symmetry-adapted blocks (the symmetric bond form
    on the orbits of the pairs) against the oracle's U(1) correlations of the
    lifted state, for the block's lowest state."""
    A = api()
    N, nup, bonds, J, perms, chi = _sym_case(case)
    basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
    ham = A.Hamiltonian(basis, J)
    storage = torch.complex128 if basis.is_complex else torch.float64
    _, psi, _ = ham.ground_state(max_iter=120, seed=2, storage=storage)
    pairs = [(0, j) for j in range(N)] + [(3, 7), (5, 5), (N - 1, 2)]
    got = basis.correlations(psi, pairs)
    st = orc.enumerate_states(N, nup)
    v = orc.SymBlock(N, nup, perms, chi).lift(st) @ psi.cpu().numpy()
    want = orc.correlations(N, st, pairs, "ss", v.real) + orc.correlations(N, st, pairs, "ss", v.imag)
    assert np.abs(got - want).max() < 1e-10
    with pytest.raises(A.XDError):
        basis.correlations(psi, pairs, "zz")

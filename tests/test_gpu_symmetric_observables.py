"""Observables of symmetry-adapted blocks on the GPU: two-point spin
correlations (the symmetric bond form on the orbits of the site pairs)
against the oracle's U(1) correlations of the lifted state, and the
finite-temperature Lanczos tridiagonals against the oracle's Lanczos on the
dense block from the same seeded starts."""
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
    """<psi|S_i.S_j|psi> and <psi|Sz_i Sz_j|psi> on symmetry-adapted blocks
    (through xd_correlations: the symmetric bond form on the orbits of the
    pairs, on the block's own representatives) against the oracle's U(1)
    correlations of the lifted state: the block's lowest state, and the same
    state scaled by 2.5 (values, i = j included, scale with <psi|psi>)."""
    A = api()
    N, nup, bonds, J, perms, chi = _sym_case(case)
    basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
    ham = A.Hamiltonian(basis, J)
    storage = torch.complex128 if basis.is_complex else torch.float64
    _, psi, _ = ham.ground_state(max_iter=120, seed=2, storage=storage)
    pairs = [(0, j) for j in range(N)] + [(3, 7), (5, 5), (N - 1, 2), (7, 3)]
    st = orc.enumerate_states(N, nup)
    lift = orc.SymBlock(N, nup, perms, chi).lift(st)
    for scale in (1.0, 2.5):
        ps = psi * scale
        v = lift @ ps.cpu().numpy()
        for kind in ("ss", "zz"):
            got = basis.correlations(ps, pairs, kind)
            want = orc.correlations(N, st, pairs, kind, v.real) + orc.correlations(N, st, pairs, kind, v.imag)
            assert np.abs(got - want).max() < 1e-10 * scale ** 2


@pytest.mark.parametrize("case", [0, 2])
def test_symmetric_block_ftlm(orc, case):
    A = api()
    N, nup, bonds, J, perms, chi = _sym_case(case)
    basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
    ham = A.Hamiltonian(basis, J)
    R, M, seed = 5, 12, 40
    a, b, n = ham.ftlm(R, M, seed)
    H = orc.SymBlock(N, nup, perms, chi).dense(bonds, J)
    if not basis.is_complex:
        H = H.real
    for r in range(R):
        start = orc.rng_normal(seed + r, 0, basis.dim)
        ao, bo = orc.lanczos(lambda v: H @ v, basis.dim, start.astype(H.dtype), M, full_reorth=False, tol=0.0)
        k = n[r]
        assert k == M == len(ao)
        assert np.abs(a[r, :k] - ao).max() <= 1e-9 * np.abs(ao).max()
        assert np.abs(b[r, :k - 1] - bo[:k - 1]).max() <= 1e-9 * np.abs(bo).max()
    # thermodynamics from longer runs: the block's ground level at low temperature
    a, b, n = ham.ftlm(4, 40, seed)
    Z, E, C = A.ftlm_thermo(a, b, n, basis.dim, [0.01])
    assert abs(E[0] - np.linalg.eigvalsh(H)[0]) < 1e-8

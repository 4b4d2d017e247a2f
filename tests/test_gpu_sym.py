"""Symmetry-adapted blocks (a4') on the GPU against the oracle."""
import math

import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def _chain(N, m):
    return N, W.chain(N), np.ones(N), W.chain_translations(N), W.chain_characters(N, m)


def _torus(Lx, Ly, mx, my):
    b, J = W.square_j1j2(Lx, Ly)
    return Lx * Ly, b, J, W.torus_translations(Lx, Ly), W.torus_characters(Lx, Ly, mx, my)


def _dihedral(N, m, parity):
    return N, W.chain(N), np.ones(N), W.chain_dihedral(N), W.chain_dihedral_characters(N, m, parity)


def _space_group(L):
    # 8 L^2 group elements: 128 at L = 4, the largest group the library takes
    b, J = W.square_j1j2(L, L)
    g = W.torus_space_group(L)
    return L * L, b, J, g, np.ones(len(g), dtype=np.complex128)


CASES = [_chain(8, 0), _chain(8, 4), _chain(10, 1), _chain(12, 3), _chain(13, 2),
         _torus(3, 3, 1, 0), _torus(4, 4, 0, 0), _torus(4, 4, 1, 2), _torus(2, 6, 1, 1),
         _dihedral(8, 0, 1), _dihedral(10, 5, -1), _dihedral(12, 0, -1), _dihedral(12, 6, 1),
         _space_group(4)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sym_basis_and_apply(orc, case):
    A = api()
    N, bonds, J, perms, chi = CASES[case]
    for nup in sorted({N // 2, max(0, N // 2 - 2)}):
        blk = orc.SymBlock(N, nup, perms, chi)
        basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
        assert basis.dim == blk.dim == orc.burnside_dim(N, nup, perms, chi)
        if blk.dim == 0:
            continue
        for k in range(blk.dim):
            assert basis.state(k) == int(blk.reps[k])
            assert basis.index(int(blk.reps[k])) == k
        ham = A.Hamiltonian(basis, J)
        rng = np.random.default_rng(case)
        x = rng.standard_normal(blk.dim) + (1j * rng.standard_normal(blk.dim) if basis.is_complex else 0)
        yo = blk.apply(bonds, J, x)
        if basis.is_complex:
            y = ham.apply(torch.from_numpy(x.astype(np.complex128)).cuda()).cpu().numpy()
        else:
            y = ham.apply(torch.from_numpy(x.real.copy()).cuda()).cpu().numpy()
            assert np.abs(yo.imag).max() < 1e-13
            yo = yo.real
        assert rel_l2(y, yo) <= 1e-12


def test_sym_lanczos_spectra_union(orc):
    A = api()
    N = 12
    bonds = W.chain(N)
    st = orc.enumerate_states(N, 6)
    full = np.linalg.eigvalsh(orc.dense_u1(N, st, bonds, np.ones(N)))
    e0s = []
    for m in range(N):
        basis = A.Basis(N, 6, bonds, symmetry=(W.chain_translations(N), W.chain_characters(N, m)))
        ham = A.Hamiltonian(basis, np.ones(N))
        storage = torch.complex128 if basis.is_complex else torch.float64
        info = ham.lanczos(max_iter=min(basis.dim, 120), seed=2, storage=storage)
        e0s.append(info["evals"][0])
    assert abs(min(e0s) - full[0]) < 1e-10 * abs(full[0])


def test_sym_gradient_matches_u1(orc):
    """Chain N=12 (N/2 even: the ground state has momentum 0)."""
    A = api()
    N = 12
    bonds = W.chain(N)
    J = np.ones(N)
    basis = A.Basis(N, 6, bonds, symmetry=(W.chain_translations(N), W.chain_characters(N, 0)))
    ham = A.Hamiltonian(basis, J)
    e0, psi, _ = ham.ground_state(max_iter=100, seed=1)
    g = ham.energy_grad(psi)
    st = orc.enumerate_states(N, 6)
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    hf = orc.bond_forms(N, st, bonds, V[:, 0], V[:, 0])
    assert w[1] - w[0] > 1e-6
    assert abs(e0 - w[0]) < 1e-10 * abs(w[0])
    assert np.abs(g - hf).max() < 1e-8


def test_sym_errors(orc):
    A = api()
    from paper_2505_02901_gb300._lib import XD_ESYM, XDError
    perms = W.chain_translations(8)
    chi = W.chain_characters(8, 1).copy()
    chi[2] = 1.0
    with pytest.raises(XDError) as e:
        A.Basis(8, 4, W.chain(8), symmetry=(perms, chi))
    assert e.value.status == XD_ESYM
    with pytest.raises(XDError) as e:
        A.Basis(8, 4, W.chain(8), symmetry=(perms[1:], W.chain_characters(8, 0)[1:]))
    assert e.value.status == XD_ESYM
    with pytest.raises(XDError) as e:  # graph not invariant
        A.Basis(8, 4, W.chain(8)[:-1], symmetry=(perms, W.chain_characters(8, 0)))
    assert e.value.status == XD_ESYM
    b = A.Basis(8, 4, W.chain(8), symmetry=(perms, W.chain_characters(8, 0)))
    with pytest.raises(XDError) as e:  # couplings not invariant
        A.Hamiltonian(b, np.arange(8.0))
    assert e.value.status == XD_ESYM

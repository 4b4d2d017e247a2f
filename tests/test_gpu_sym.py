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
    # 8 L^2 group elements (128 at L = 4)
    b, J = W.square_j1j2(L, L)
    g = W.torus_space_group(L)
    return L * L, b, J, g, np.ones(len(g), dtype=np.complex128)


# tori: rows of up to 7 sites take the row-state search with its row-step
# table; 8 sites (8x2) the narrowing from the word; more than 8 rows (2x9)
# the scan over the translations reaching the smallest top row
CASES = [_chain(8, 0), _chain(8, 4), _chain(10, 1), _chain(12, 3), _chain(13, 2),
         _torus(3, 3, 1, 0), _torus(4, 4, 0, 0), _torus(4, 4, 1, 2), _torus(2, 6, 1, 1),
         _torus(8, 2, 1, 1), _torus(8, 2, 0, 0), _torus(2, 9, 1, 3),
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


def _wide(Lx, Ly, lattice, r, m, mx=0, my=0):
    if lattice == "triangular":
        b, J = W.triangular(Lx)
    else:
        b, J = W.square_j1j2(Lx, Ly)
    return (Lx * Ly, b, J, W.space_group(Lx, Ly, lattice),
            W.space_group_characters(Lx, Ly, lattice, r, m, mx, my))


def _mirror_translations(Lx, Ly, m, my):
    """Translations times the single mirror x -> -x (elements R^0 M^e of the
    rectangular group): every ky is invariant, so the characters are complex."""
    b, J = W.square_j1j2(Lx, Ly)
    g = W.space_group(Lx, Ly, "rectangular")
    c = W.space_group_characters(Lx, Ly, "rectangular", 1, m, 0, my)
    T = Lx * Ly
    rows = np.r_[0:T, 2 * T:3 * T]
    return Lx * Ly, b, J, g[rows], c[rows]


def _scrambled(case, seed):
    N, b, J, g, c = case
    p = np.random.default_rng(seed).permutation(len(g))
    return N, b, J, g[p], c[p]


# (case, sectors): 96 to 432 group elements, translations times C2v, C4v, C6v
WIDE = [
    (_wide(3, 3, "triangular", 1, 1), (3, 4, 5)),
    (_wide(3, 3, "triangular", -1, -1), (4,)),
    (_wide(4, 4, "triangular", 1, -1), (5, 6)),
    (_wide(3, 4, "rectangular", -1, 1, 0, 2), (5, 6)),
    (_wide(4, 6, "rectangular", 1, 1, 2, 3), (4,)),
    (_wide(5, 5, "square", -1, 1), (4,)),
    (_wide(6, 6, "square", 1, 1), (3, 4)),
    (_wide(6, 6, "square", -1, -1, 3, 3), (4,)),
    (_wide(6, 6, "triangular", 1, 1), (3,)),
    (_mirror_translations(4, 6, -1, 1), (4, 5)),
    (_scrambled(_wide(4, 4, "triangular", 1, 1), 3), (5,)),
    (_scrambled(_mirror_translations(3, 4, 1, 1), 5), (6,)),
]


@pytest.mark.parametrize("case", range(len(WIDE)))
def test_wide_groups_basis_and_apply(orc, case):
    """Space groups beyond 128 elements take the translation-coset orbit
    search: representatives, |Stab| through the products, and y = H x match the
    oracle's plain search over every group element."""
    A = api()
    (N, bonds, J, perms, chi), sectors = WIDE[case]
    for nup in sectors:
        blk = orc.SymBlock(N, nup, perms, chi)
        basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
        assert basis.dim == blk.dim == orc.burnside_dim(N, nup, perms, chi)
        if blk.dim == 0:
            continue
        got = np.array([basis.state(k) for k in range(blk.dim)], dtype=np.uint64)
        assert np.array_equal(got, blk.reps)
        ham = A.Hamiltonian(basis, J)
        rng = np.random.default_rng(case * 10 + nup)
        if basis.is_complex:
            x = rng.standard_normal(blk.dim) + 1j * rng.standard_normal(blk.dim)
            y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        else:
            x = rng.standard_normal(blk.dim)
            y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        yo = blk.apply(bonds, J, x)
        if not basis.is_complex:
            assert np.abs(yo.imag).max() < 1e-13
            yo = yo.real
        assert rel_l2(y, yo) <= 1e-12


def test_wide_group_bilinear_and_limit(orc):
    """Bond forms on a 192-element block against the oracle's U(1) forms of
    the lifted vectors, and the group-size limit."""
    A = api()
    from paper_2505_02901_gb300._lib import XDError
    N, bonds, J, perms, chi = _wide(4, 4, "triangular", 1, 1)
    nup = 6
    blk = orc.SymBlock(N, nup, perms, chi)
    basis = A.Basis(N, nup, bonds, symmetry=(perms, chi))
    ham = A.Hamiltonian(basis, J)
    rng = np.random.default_rng(11)
    g = rng.standard_normal(blk.dim)
    x = rng.standard_normal(blk.dim)
    st = orc.enumerate_states(N, nup)
    B = blk.lift(st)
    want = orc.bond_forms(N, st, bonds, (B @ g).real, (B @ x).real)
    # within a one-dimensional irrep the form is constant on each bond orbit
    # (one orbit here: every bond of the triangular lattice)
    assert np.ptp(want) < 1e-11 * max(1.0, np.abs(want).max())
    got = ham.bilinear(torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())
    big = np.tile(perms, (11, 1))[:2049]
    with pytest.raises(XDError):
        A.Basis(N, nup, bonds, symmetry=(big, np.ones(len(big), dtype=np.complex128)))

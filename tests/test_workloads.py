"""The seeded input generators: bond lists with the right counts, degrees and
no repeated pair; groups that are closed, contain the identity and list
every element once; characters that are homomorphisms; reproducible
batches.  (The generators hold no arithmetic of the method; these checks
keep every parity test's inputs what their names say.)"""
import math

import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W


def _degrees(bonds, N):
    d = np.zeros(N, dtype=int)
    for i, j in bonds:
        d[i] += 1
        d[j] += 1
    return d


def _pairs(bonds):
    return {(min(int(i), int(j)), max(int(i), int(j))) for i, j in bonds}


@pytest.mark.parametrize("N", [2, 3, 8, 13])
def test_chain(N):
    b = W.chain(N)
    assert len(_pairs(b)) == len(b) == (1 if N == 2 else N)


def test_j1j2_chain_and_ladder():
    b, J = W.chain_j1j2(10)
    assert len(_pairs(b)) == 20 and (_degrees(b, 10) == 4).all() and (J[:10] == 1).all() and (J[10:] == 0.5).all()
    lad = W.ladder(14, 2)
    assert len(lad) == 56 and len(_pairs(lad)) == 42  # each rung listed twice
    assert len(W.ladder(14, 1)) == 42


@pytest.mark.parametrize("Lx,Ly,nb", [(4, 8, 128), (6, 6, 144), (4, 4, 64), (4, 6, 96)])
def test_square_j1j2(Lx, Ly, nb):
    b, J = W.square_j1j2(Lx, Ly)
    N = Lx * Ly
    assert len(b) == nb == len(_pairs(b))
    assert (_degrees(b, N) == 8).all()
    assert np.count_nonzero(J == 1.0) == nb // 2


@pytest.mark.parametrize("L", [3, 4, 6])
def test_triangular(L):
    b, J = W.triangular(L)
    assert len(b) == 3 * L * L == len(_pairs(b))
    assert (_degrees(b, L * L) == 6).all()


@pytest.mark.parametrize("Lx,Ly,lattice,order", [(4, 4, "square", 128), (6, 6, "square", 288),
                                                 (3, 3, "triangular", 108), (6, 6, "triangular", 432),
                                                 (4, 6, "rectangular", 96), (3, 4, "rectangular", 48)])
def test_space_groups_are_groups(orc, Lx, Ly, lattice, order):
    g = W.space_group(Lx, Ly, lattice)
    N = Lx * Ly
    assert g.shape == (order, N)
    assert (g[0] == np.arange(N)).all()  # identity first
    assert len({tuple(r) for r in g.tolist()}) == order  # every element once
    assert orc.group_check(N, g) == 0  # permutations, closed, inverses
    for r in (1, -1):
        for m in (1, -1):
            assert orc.group_check(N, g, W.space_group_characters(Lx, Ly, lattice, r, m)) == 0
    # the bond graph of the lattice is mapped onto itself
    b = (W.triangular(Lx)[0] if lattice == "triangular" else W.square_j1j2(Lx, Ly)[0])
    E = _pairs(b)
    for row in g:
        assert {(min(row[i], row[j]), max(row[i], row[j])) for i, j in E} == E


def test_space_group_momentum_must_be_invariant(orc):
    """(pi, pi) is invariant under C4v and gives a homomorphism; (pi/2, 0) is
    not, and the group check says so."""
    g = W.space_group(4, 4, "square")
    assert orc.group_check(16, g, W.space_group_characters(4, 4, "square", 1, 1, 2, 2)) == 0
    assert orc.group_check(16, g, W.space_group_characters(4, 4, "square", 1, 1, 1, 0)) != 0
    with pytest.raises(ValueError):
        W.space_group(4, 6, "square")


def test_translation_and_dihedral_characters(orc):
    for Lx, Ly in ((4, 4), (2, 6), (6, 6)):
        T = W.torus_translations(Lx, Ly)
        for mx in range(Lx):
            assert orc.group_check(Lx * Ly, T, W.torus_characters(Lx, Ly, mx, (mx + 1) % Ly)) == 0
    for N in (8, 9, 12):
        assert orc.group_check(N, W.chain_translations(N), W.chain_characters(N, 1)) == 0
    D = W.chain_dihedral(12)
    for m in (0, 6):
        for p in (1, -1):
            assert orc.group_check(12, D, W.chain_dihedral_characters(12, m, p)) == 0
    with pytest.raises(ValueError):
        W.chain_dihedral_characters(12, 1, 1)


def test_batched_instances_are_reproducible():
    a, b = W.batched_instances(16, seed=4), W.batched_instances(16, seed=4)
    assert all(x["N"] == y["N"] and np.array_equal(x["J"], y["J"]) for x, y in zip(a, b))
    assert all(d["N"] in (18, 20, 22, 24, 26, 28) and d["nup"] == d["N"] // 2 for d in a)
    assert all(len(d["bonds"]) == (d["N"] if d["kind"] == "chain" else 2 * d["N"]) for d in a)
    assert len({d["kind"] for d in W.batched_instances(64, seed=4)}) == 2
    J = W.uniform_couplings(1000, 3)
    assert J.min() >= 0.5 and J.max() < 1.5 and math.isclose(J.mean(), 1.0, abs_tol=0.05)

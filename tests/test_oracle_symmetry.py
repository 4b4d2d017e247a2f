"""Pins of the oracle's symmetry-adapted blocks (Sec. 3.9, Sec. 3.10)."""
import math
import os

import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _toml_group():
    perms, chis = [], {}
    for line in open(os.path.join(GOLD, "sym_c4_toml.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "perm":
            perms.append([int(v) for v in t[1:]])
        else:
            v = [float(a) for a in t[1:]]
            chis[t[0]] = np.array([complex(v[2 * i], v[2 * i + 1]) for i in range(len(v) // 2)])
    return np.array(perms, dtype=np.int32), chis


def test_paper_worked_example(orc):
    perms, chis = _toml_group()
    st = orc.enumerate_states(4, 2)
    v = orc.project(4, perms, chis["pi"], 0b1100, st)
    ref = {}
    for line in open(os.path.join(GOLD, "sym_c4_kpi.txt")):
        t = line.split()
        if t and not t[0].startswith("#"):
            ref[int(t[0])] = float(t[1])
    expect = np.zeros(st.size, dtype=np.complex128)
    for w, c in ref.items():
        expect[orc.index_search(st, w)] = c
    assert np.abs(v - expect).max() < 1e-15


def test_toml_representations_are_valid(orc):
    perms, chis = _toml_group()
    assert orc.group_check(4, perms) == 0
    for name in ("zero", "pihalf", "pi"):
        assert orc.group_check(4, perms, chis[name]) == 0


def test_group_axiom_failures(orc):
    perms, chis = _toml_group()
    assert orc.group_check(4, perms[1:]) == 2                 # no identity
    assert orc.group_check(4, perms[[0, 1]]) == 3             # not closed
    bad = perms.copy(); bad[1] = [0, 0, 1, 2]
    assert orc.group_check(4, bad) == 1                       # not a permutation
    chi = chis["pihalf"].copy(); chi[2] = 1.0
    assert orc.group_check(4, perms, chi) == 5                # not a homomorphism
    assert orc.group_check(4, perms, 2 * chis["zero"]) in (5, 6)


CASES = [("chain", 8, None), ("chain", 10, None), ("torus", 2, 4), ("torus", 3, 3)]


def _case(kind, a, b):
    if kind == "chain":
        return a, W.chain(a), np.ones(a), W.chain_translations(a), \
            [W.chain_characters(a, m) for m in range(a)]
    bonds, J = W.square_j1j2(a, b, 1.0, 0.5)
    return a * b, bonds, J, W.torus_translations(a, b), \
        [W.torus_characters(a, b, mx, my) for my in range(b) for mx in range(a)]


@pytest.mark.parametrize("kind,a,b", CASES)
def test_dims_burnside_and_sum(orc, kind, a, b):
    N, bonds, J, perms, chis = _case(kind, a, b)
    for nup in range(N + 1):
        dims = []
        for chi in chis:
            blk = orc.SymBlock(N, nup, perms, chi)
            assert blk.dim == orc.burnside_dim(N, nup, perms, chi)
            assert np.all(np.diff(blk.reps.astype(np.int64)) > 0)
            dims.append(blk.dim)
        assert sum(dims) == math.comb(N, nup)


@pytest.mark.parametrize("kind,a,b", CASES)
def test_symmetric_matrix_equals_projection(orc, kind, a, b):
    N, bonds, J, perms, chis = _case(kind, a, b)
    nup = N // 2
    st = orc.enumerate_states(N, nup)
    H = orc.dense_u1(N, st, bonds, J)
    spec = []
    for chi in chis:
        blk = orc.SymBlock(N, nup, perms, chi)
        if blk.dim == 0:
            continue
        B = blk.lift(st)
        assert np.abs(B.conj().T @ B - np.eye(blk.dim)).max() < 1e-13
        Hk = blk.dense(bonds, J)
        assert np.abs(Hk - B.conj().T @ H @ B).max() < 1e-13
        assert np.abs(Hk - Hk.conj().T).max() < 1e-14
        spec.append(np.linalg.eigvalsh(Hk))
    # union of the momentum spectra is the U(1) spectrum
    assert np.abs(np.sort(np.concatenate(spec)) - np.linalg.eigvalsh(H)).max() < 1e-11


def test_lifted_eigenvector_has_its_momentum(orc):
    N = 10
    bonds, perms = W.chain(N), W.chain_translations(N)
    st = orc.enumerate_states(N, 5)
    T = np.zeros((st.size, st.size))
    for k, s in enumerate(st):
        T[orc.index_search(st, orc.act(N, perms[1], int(s))), k] = 1.0
    for m in (0, 1, 3):
        chi = W.chain_characters(N, m)
        blk = orc.SymBlock(N, 5, perms, chi)
        w, V = np.linalg.eigh(blk.dense(bonds, np.ones(N)))
        psi = blk.lift(st) @ V[:, 0]
        assert np.abs(T @ psi - chi[1] * psi).max() < 1e-12


def test_burnside_6x6_momentum_sectors(orc):
    perms = W.torus_translations(6, 6)
    assert orc.burnside_dim(36, 18, perms, W.torus_characters(6, 6, 0, 0)) == 252091362
    assert orc.burnside_dim(36, 18, perms, W.torus_characters(6, 6, 1, 0)) == 252085716
    total = sum(orc.burnside_dim(36, 18, perms, W.torus_characters(6, 6, mx, my))
                for mx in range(6) for my in range(6))
    assert total == math.comb(36, 18)


@pytest.mark.parametrize("N", [8, 10])
def test_dihedral_blocks(orc, N):
    """D_N (translations and reflections): every one-dimensional irrep block is
    the projection of H, and its spectrum lies inside the U(1) spectrum."""
    bonds, J, perms = W.chain(N), np.ones(N), W.chain_dihedral(N)
    nup = N // 2
    st = orc.enumerate_states(N, nup)
    H = orc.dense_u1(N, st, bonds, J)
    ev = np.linalg.eigvalsh(H)
    total = 0
    for m in (0, N // 2):
        for parity in (1, -1):
            chi = W.chain_dihedral_characters(N, m, parity)
            blk = orc.SymBlock(N, nup, perms, chi)
            assert blk.dim == orc.burnside_dim(N, nup, perms, chi)
            total += blk.dim
            if blk.dim == 0:
                continue
            B = blk.lift(st)
            assert np.abs(B.conj().T @ B - np.eye(blk.dim)).max() < 1e-13
            Hk = blk.dense(bonds, J)
            assert np.abs(Hk - B.conj().T @ H @ B).max() < 1e-13
            for e in np.linalg.eigvalsh(Hk):
                assert np.abs(ev - e).min() < 1e-11
    # the one-dimensional irreps do not exhaust the block (D_N has 2-d irreps)
    assert 0 < total < math.comb(N, nup)


def test_space_group_4x4_block(orc):
    """The 128-element space group of the 4x4 square lattice, trivial irrep:
    the block's product equals the projected U(1) product on random vectors,
    and its lowest level is the ground state of the whole Sz = 0 block."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    bonds, J = W.square_j1j2(4, 4)
    perms = W.torus_space_group(4)
    chi = np.ones(len(perms), dtype=np.complex128)
    st = orc.enumerate_states(16, 8)
    blk = orc.SymBlock(16, 8, perms, chi)
    assert blk.dim == orc.burnside_dim(16, 8, perms, chi)
    B = blk.lift(st)
    assert np.abs(B.conj().T @ B - np.eye(blk.dim)).max() < 1e-13
    rng = np.random.default_rng(7)
    for _ in range(3):
        x = rng.standard_normal(blk.dim)
        hx = B.conj().T @ orc.apply_u1(16, st, bonds, J, (B @ x).real)
        assert np.abs(blk.apply(bonds, J, x) - hx).max() < 1e-12
    op = LinearOperator((st.size, st.size), matvec=lambda v: orc.apply_u1(16, st, bonds, J, v))
    e0 = eigsh(op, k=1, which="SA", tol=1e-12)[0][0]
    # the ground state of the frustrated 4x4 J1-J2 model (J2 = 0.5) is fully symmetric
    assert abs(np.linalg.eigvalsh(blk.dense(bonds, J))[0] - e0) < 1e-9


def test_dihedral_chain36_dimension(orc):
    """N = 36 chain, Sz = 0, translations and reflections, trivial irrep: the
    sector of the paper's U(1) + lattice benchmark, quoted there as dim 1.3e8."""
    perms = W.chain_dihedral(36)
    chi = W.chain_dihedral_characters(36, 0, 1)
    d = orc.burnside_dim(36, 18, perms, chi)
    assert d == 126068558
    assert abs(d - 1.3e8) / 1.3e8 < 0.05
    # N = 40, quoted as dim 1.7e9
    d40 = orc.burnside_dim(40, 20, W.chain_dihedral(40), W.chain_dihedral_characters(40, 0, 1))
    assert d40 == 1723176308
    assert abs(d40 - 1.7e9) / 1.7e9 < 0.05


SPACE_GROUPS = [(3, 3, "triangular", 4), (4, 4, "triangular", 5), (3, 4, "rectangular", 6),
                (4, 6, "rectangular", 3), (5, 5, "square", 3)]


@pytest.mark.parametrize("Lx,Ly,lattice,nup", SPACE_GROUPS)
def test_space_group_blocks_are_projections(orc, Lx, Ly, lattice, nup):
    """Translations times the point group (C6v, C2v, C4v; 108 to 200 elements)
    at Gamma, all four one-dimensional irreps: the block is the projection of
    the U(1) block (orthonormal lifted columns, product equal to the projected
    U(1) product on random vectors) and every eigenvector of the block lifts to
    an eigenvector of the U(1) Hamiltonian with the same energy."""
    N = Lx * Ly
    if lattice == "triangular":
        bonds, J = W.triangular(Lx)
    else:
        bonds, J = W.square_j1j2(Lx, Ly)
    perms = W.space_group(Lx, Ly, lattice)
    st = orc.enumerate_states(N, nup)
    rng = np.random.default_rng(N)
    total = 0
    for r in (1, -1):
        for m in (1, -1):
            chi = W.space_group_characters(Lx, Ly, lattice, r, m)
            blk = orc.SymBlock(N, nup, perms, chi)
            assert blk.dim == orc.burnside_dim(N, nup, perms, chi)
            total += blk.dim
            if blk.dim == 0:
                continue
            B = blk.lift(st)
            assert np.abs(B.conj().T @ B - np.eye(blk.dim)).max() < 1e-13
            for _ in range(2):
                x = rng.standard_normal(blk.dim) + 1j * rng.standard_normal(blk.dim)
                Bx = B @ x
                hx = orc.apply_u1(N, st, bonds, J, Bx.real) + 1j * orc.apply_u1(N, st, bonds, J, Bx.imag)
                assert np.abs(blk.apply(bonds, J, x) - B.conj().T @ hx).max() < 1e-12
            Hk = blk.dense(bonds, J)
            assert np.abs(Hk - Hk.conj().T).max() < 1e-13
            w, V = np.linalg.eigh(Hk)
            for k in range(min(3, blk.dim)):
                psi = B @ V[:, k]
                hp = orc.apply_u1(N, st, bonds, J, psi.real) + 1j * orc.apply_u1(N, st, bonds, J, psi.imag)
                assert np.abs(hp - w[k] * psi).max() < 1e-11
    assert 0 < total <= math.comb(N, nup)


def test_space_group_6x6_dimensions(orc):
    """Burnside dimensions of the 288-element square and 432-element
    triangular space groups of the 36-site tori at Sz = 0, trivial irrep: the
    two blocks are about 1/|G| of C(36, 18), and the 2-d irreps keep the
    one-dimensional blocks of the square group short of the full count."""
    sq = W.space_group(6, 6, "square")
    tri = W.space_group(6, 6, "triangular")
    d_sq = orc.burnside_dim(36, 18, sq, W.space_group_characters(6, 6, "square"))
    d_tri = orc.burnside_dim(36, 18, tri, W.space_group_characters(6, 6, "triangular"))
    full = math.comb(36, 18)
    assert abs(d_sq * 288 / full - 1) < 0.01 and abs(d_tri * 432 / full - 1) < 0.01
    gamma = sum(orc.burnside_dim(36, 18, sq, W.space_group_characters(6, 6, "square", r, m))
                for r in (1, -1) for m in (1, -1))
    assert gamma < orc.burnside_dim(36, 18, W.torus_translations(6, 6), W.torus_characters(6, 6, 0, 0))


def test_keyed_values_agree_everywhere(orc):
    """The keyed input generator: the oracle's C definition, the numpy and
    the torch implementations of workloads.py give identical bits."""
    torch = pytest.importorskip("torch")
    w = np.array([0, 1, 2, 3, 12345, 2**35 + 11, 2**40 - 7], dtype=np.uint64)
    for seed in (0, 7, 2**63 + 5):
        a = orc.keyed(seed, w, True)
        b = W.keyed_values(seed, w, True)
        c = W.keyed_values_torch(seed, torch.from_numpy(w.astype(np.int64)), True).numpy()
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.all(np.abs(a.real) <= 1) and np.all(np.abs(a.imag) <= 1)


@pytest.mark.parametrize("kind,a,b", CASES)
def test_sampled_rows_keyed_equal_the_projected_block(orc, kind, a, b):
    """Rows of the symmetric product for a vector keyed on the
    representatives, computed from the representatives alone (membership test
    and keyed values instead of a list), equal the rows of B^H H B x with B
    the lifted basis of the projector (Sec. 3.10), for every momentum."""
    N, bonds, J, perms, chis = _case(kind, a, b)
    nup = N // 2
    st = orc.enumerate_states(N, nup)
    H = orc.dense_u1(N, st, bonds, J)
    for chi in chis:
        blk = orc.SymBlock(N, nup, perms, chi)
        if blk.dim == 0:
            continue
        cplx = bool(np.abs(np.imag(chi)).max() > 1e-12)
        B = blk.lift(st)
        x = orc.keyed(5, blk.reps, cplx)
        y = B.conj().T @ H @ B @ x
        yr = orc.sym_apply_rows_keyed(N, perms, chi, bonds, J, 5, cplx, blk.reps)
        assert np.abs(yr - y).max() <= 1e-13 * max(1.0, np.abs(y).max())


def test_sampled_rows_keyed_equal_the_full_product_4x4(orc):
    """4x4 J1-J2 with its 16 translations (and the 128-element space group at
    Gamma, where targets whose representative leaves the block drop out):
    sampled rows by representatives equal the full symmetric product."""
    bonds, J = W.square_j1j2(4, 4)
    groups = [(W.torus_translations(4, 4), W.torus_characters(4, 4, mx, my)) for mx, my in ((0, 0), (1, 0), (2, 2))]
    groups.append((W.torus_space_group(4), None))
    for perms, chi in groups:
        if chi is None:
            chi = np.ones(len(perms))
        blk = orc.SymBlock(16, 8, perms, chi)
        cplx = bool(np.abs(np.imag(chi)).max() > 1e-12)
        x = orc.keyed(9, blk.reps, cplx)
        y = blk.apply(bonds, J, x)
        rows = np.random.default_rng(3).choice(blk.dim, min(200, blk.dim), replace=False)
        yr = orc.sym_apply_rows_keyed(16, perms, chi, bonds, J, 9, cplx, blk.reps[rows])
        assert np.abs(yr - y[rows]).max() <= 1e-13 * np.abs(y).max()

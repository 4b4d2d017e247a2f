"""Full-size checks of the benchmark workloads on the GPU.

Where the oracle cannot run the whole product, parity is checked on sampled
rows (counting index, seeded vector regenerated on the CPU) and through
properties that hold at any size: Burnside dimensions, valid ascending
representatives, Hermiticity, agreement of energies between independent
forms of the product, Euler's identity and finite differences."""
import math

import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def test_c5b_square6x6_u1_sampled_rows(orc):
    """6x6 J1-J2, Sz=0 without symmetry: dim 9,075,135,300 (int64 rows), FP32."""
    A = api()
    bonds, J = W.square_j1j2(6, 6)
    ham = A.Hamiltonian(A.Basis(36, 18, bonds), J)
    assert ham.dim == math.comb(36, 18) == 9075135300
    seed = 6
    x = A.random_vector(ham.dim, seed, torch.float32)
    y = ham.apply(x)
    del x
    rows = np.concatenate([[0, ham.dim - 1, 2**32 + 5], np.random.default_rng(6).integers(0, ham.dim, 300)])
    yo = orc.apply_rows_rng(36, 18, bonds, J, seed, rows)
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert rel_l2(ys, yo) <= 5e-6
    del y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("mx", [0, 1])
def test_c5a_square6x6_sampled_rows(orc, mx):
    """6x6 J1-J2 with its 36 translations at k=(0,0) (real FP64) and
    k=(pi/3,0) (complex128), ~2.5e8 representatives each, at full size:
    x keyed on each row's representative word (the block's words from
    xd_basis_states), y = H x on the GPU; sampled rows (first, last and 3000
    random ones) against the oracle's row formula of the projector (Sec. 3.10)
    evaluated from the representatives alone, relative L2 <= 1e-12; every
    sampled word a valid representative of the block."""
    A = api()
    bonds, J = W.square_j1j2(6, 6)
    perms, chi = W.torus_translations(6, 6), W.torus_characters(6, 6, mx, 0)
    basis = A.Basis(36, 18, bonds, symmetry=(perms, chi))
    assert basis.dim == (252091362 if mx == 0 else 252085716)
    ham = A.Hamiltonian(basis, J)
    seed = 40 + mx
    x = W.keyed_values_torch(seed, basis.states(), basis.is_complex)
    y = ham.apply(x)
    del x
    rows = np.concatenate([[0, basis.dim - 1], np.random.default_rng(10 + mx).integers(0, basis.dim, 3000)])
    rt = torch.from_numpy(rows).cuda()
    words = basis.states()[rt].cpu().numpy().astype(np.uint64)
    ys = y[rt].cpu().numpy()
    del y
    torch.cuda.empty_cache()
    for k in (0, 1, 2, 500, 2999):
        r, u, cnt = orc.rep(36, perms, int(words[k]))
        assert r == int(words[k])
    yo = orc.sym_apply_rows_keyed(36, perms, chi, bonds, J, seed, basis.is_complex, words)
    if not basis.is_complex:
        yo = yo.real
    assert rel_l2(ys, yo) <= 1e-12
    assert np.abs(ys - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("mx", [0, 1])
def test_c5a_square6x6_momentum_blocks(orc, mx):
    """6x6 J1-J2 with its 36 translations at k=(0,0) (real) and k=(pi/3,0)
    (complex): Burnside dimension, sampled representatives valid and
    ascending, and <u, H v> = conj <v, H u> at full size."""
    A = api()
    bonds, J = W.square_j1j2(6, 6)
    perms, chi = W.torus_translations(6, 6), W.torus_characters(6, 6, mx, 0)
    basis = A.Basis(36, 18, bonds, symmetry=(perms, chi))
    assert basis.dim == orc.burnside_dim(36, 18, perms, chi)
    assert basis.dim == (252091362 if mx == 0 else 252085716)
    rng = np.random.default_rng(mx)
    for k in np.concatenate([[0, basis.dim - 2], rng.integers(0, basis.dim - 1, 40)]):
        s, s2 = basis.state(int(k)), basis.state(int(k) + 1)
        assert s < s2
        r, u, cnt = orc.rep(36, perms, s)
        assert r == s
        stab = [g for g in range(36) if orc.act(36, perms[g], s) == s]
        assert abs(sum(chi[g] for g in stab)) > 0.5 and len(stab) == cnt
        assert basis.index(s) == k
    ham = A.Hamiltonian(basis, J)
    dt = torch.complex128 if basis.is_complex else torch.float64
    g = torch.Generator(device="cuda").manual_seed(7)
    u = torch.randn(basis.dim, dtype=dt, device="cuda", generator=g)
    v = torch.randn(basis.dim, dtype=dt, device="cuda", generator=g)
    uhv = torch.vdot(u, ham.apply(v)).item()
    vhu = torch.vdot(v, ham.apply(u)).item()
    assert abs(uhv - np.conj(vhu)) <= 1e-10 * abs(uhv)


def test_c2_square4x8_lanczos_forms_agree(orc):
    """4x8 J1-J2, 200 Lanczos steps: FP32 vector storage (FP64-class dots)
    against the FP64 form; the ground energies agree to 1e-6 relative."""
    A = api()
    bonds, J = W.square_j1j2(4, 8)
    ham = A.Hamiltonian(A.Basis(32, 16, bonds), J)
    e64 = ham.lanczos(max_iter=200, seed=2, storage=torch.float64, nev=2)
    e32 = ham.lanczos(max_iter=200, seed=2, storage=torch.float32, nev=2)
    E64, E32 = e64["evals"][0], e32["evals"][0]
    assert -0.55 * 32 < E64 < -0.45 * 32
    assert abs(E32 - E64) <= 1e-6 * abs(E64)
    # converged energy; the residual estimate of the lowest Ritz pair is
    # blurred by its ghost copy (no reorthogonalisation), so it is looser
    assert e64["resid"][0] < 1e-5


def test_c3_ladder28_gradient(orc):
    """14-rung ladder, 56 bonds, J ~ U[0.5, 1.5): dE0/dJ by the backward
    kernel against central differences (h = 1e-5) on two bonds, Euler's
    identity, and equal derivatives of the two copies of every rung."""
    A = api()
    bonds = W.ladder(14, 2)
    J = W.uniform_couplings(56, 3)
    ham = A.Hamiltonian(A.Basis(28, 14, bonds), J)
    e0, psi, info = ham.ground_state(max_iter=200, seed=3)
    g = ham.energy_grad(psi)
    assert abs(J @ g - e0) <= 1e-8 * abs(e0)
    assert np.abs(g[28:42] - g[42:56]).max() < 1e-7
    h = 1e-5
    for b in (0, 30):
        Jp, Jm = J.copy(), J.copy()
        Jp[b] += h
        Jm[b] -= h
        ham.set_couplings(Jp)
        ep = ham.lanczos(max_iter=200, seed=3)["evals"][0]
        ham.set_couplings(Jm)
        em = ham.lanczos(max_iter=200, seed=3)["evals"][0]
        assert abs((ep - em) / (2 * h) - g[b]) < 1e-5
    ham.set_couplings(J)


def test_paper_chain36_u1_and_dihedral_sector(orc):
    """The paper's N=36 chain benchmarks: the U(1) block (dim 9,075,135,300,
    FP32 prefix-block product at P = 24) on sampled rows against the oracle;
    the D_36 fully symmetric block (dim 126,068,558 by Burnside, ring path of
    the orbit search) with valid ascending representatives and Hermiticity;
    and the lowest energy of that block equal to the U(1) ground energy (the
    chain's ground state at N = 36 is translation and reflection invariant)."""
    A = api()
    N = 36
    bonds, J = W.chain(N), np.ones(N)
    ham = A.Hamiltonian(A.Basis(N, N // 2, bonds), J)
    seed = 11
    x = A.random_vector(ham.dim, seed, torch.float32)
    y = ham.apply(x)
    del x
    rows = np.concatenate([[0, ham.dim - 1], np.random.default_rng(9).integers(0, ham.dim, 300)])
    yo = orc.apply_rows_rng(N, N // 2, bonds, J, seed, rows)
    assert rel_l2(y[torch.from_numpy(rows).cuda()].double().cpu().numpy(), yo) <= 5e-6
    del y
    torch.cuda.empty_cache()
    # FP32 vector storage (FP64-class dots) keeps this run near 30 s
    e_u1 = ham.lanczos(max_iter=120, seed=1, storage=torch.float32)["evals"][0]
    torch.cuda.empty_cache()

    perms, chi = W.chain_dihedral(N), W.chain_dihedral_characters(N, 0, 1)
    sym = A.Basis(N, N // 2, bonds, symmetry=(perms, chi))
    assert sym.dim == orc.burnside_dim(N, N // 2, perms, chi) == 126068558
    rng = np.random.default_rng(3)
    for k in np.concatenate([[0, sym.dim - 2], rng.integers(0, sym.dim - 1, 30)]):
        s, s2 = sym.state(int(k)), sym.state(int(k) + 1)
        assert s < s2
        r, u, cnt = orc.rep(N, perms, s)
        assert r == s
    hs = A.Hamiltonian(sym, J)
    g = torch.Generator(device="cuda").manual_seed(5)
    u = torch.randn(sym.dim, dtype=torch.float64, device="cuda", generator=g)
    v = torch.randn(sym.dim, dtype=torch.float64, device="cuda", generator=g)
    uhv = float(torch.dot(u, hs.apply(v)))
    vhu = float(torch.dot(v, hs.apply(u)))
    assert abs(uhv - vhu) <= 1e-10 * abs(uhv)
    del u, v
    e_sym = hs.lanczos(max_iter=120, seed=1)["evals"][0]
    assert abs(e_sym - e_u1) <= 1e-7 * abs(e_u1)


def test_space_groups_6x6_full_size(orc):
    """36-site tori at Sz = 0 with their full space groups: 288 elements on
    the square lattice, 432 on the triangular one (coset orbit search).
    Burnside dimensions, sampled representatives valid and ascending with
    their stabilisers, Hermiticity, and for the square Heisenberg model
    (J2 = 0) the lowest level of the fully symmetric block equal to the lowest
    level of the k = 0 translation block: with N/2 = 18 even the ground state
    is invariant under translations, and the point operations that keep the
    sublattices (all of them here) fix it by the Marshall sign rule."""
    A = api()
    for lattice in ("square", "triangular"):
        if lattice == "square":
            bonds, _ = W.square_j1j2(6, 6)
            bonds = bonds[:72]  # nearest neighbours only
        else:
            bonds, _ = W.triangular(6)
        J = np.ones(len(bonds))
        perms = W.space_group(6, 6, lattice)
        chi = W.space_group_characters(6, 6, lattice)
        sym = A.Basis(36, 18, bonds, symmetry=(perms, chi))
        assert sym.dim == orc.burnside_dim(36, 18, perms, chi)
        rng = np.random.default_rng(len(perms))
        for k in np.concatenate([[0, sym.dim - 2], rng.integers(0, sym.dim - 1, 25)]):
            s, s2 = sym.state(int(k)), sym.state(int(k) + 1)
            assert s < s2
            r, u, cnt = orc.rep(36, perms, s)
            assert r == s
            stab = [g for g in range(len(perms)) if orc.act(36, perms[g], s) == s]
            assert abs(sum(chi[g] for g in stab)) > 0.5 and len(stab) == cnt
            assert sym.index(s) == k
        hs = A.Hamiltonian(sym, J)
        g = torch.Generator(device="cuda").manual_seed(len(perms))
        u = torch.randn(sym.dim, dtype=torch.float64, device="cuda", generator=g)
        v = torch.randn(sym.dim, dtype=torch.float64, device="cuda", generator=g)
        uhv = float(torch.dot(u, hs.apply(v)))
        vhu = float(torch.dot(v, hs.apply(u)))
        assert abs(uhv - vhu) <= 1e-10 * abs(uhv)
        del u, v
        if lattice == "square":
            e_sg = hs.lanczos(max_iter=110, seed=1)["evals"][0]
            del hs, sym
            tperms, tchi = W.torus_translations(6, 6), W.torus_characters(6, 6, 0, 0)
            ht = A.Hamiltonian(A.Basis(36, 18, bonds, symmetry=(tperms, tchi)), J)
            e_t = ht.lanczos(max_iter=110, seed=1)["evals"][0]
            del ht
            assert abs(e_sg - e_t) <= 1e-9 * abs(e_t)
        torch.cuda.empty_cache()

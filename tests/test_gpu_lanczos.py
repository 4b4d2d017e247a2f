"""Lanczos (a6, a7), bilinear forms and gradients (a8) against the oracle."""
import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def test_chain16_lanczos_f64_and_f32(orc):
    """C1 workload: periodic N=16 chain, Sz=0, 100 steps."""
    A = api()
    N = 16
    bonds = W.chain(N)
    st = orc.enumerate_states(N, 8)
    ham = A.Hamiltonian(A.Basis(N, 8, bonds), np.ones(N))
    v0 = orc.rng_normal(1, 0, st.size)
    a, b = orc.lanczos(lambda v: orc.apply_u1(N, st, bonds, np.ones(N), v), st.size, v0, 100)
    e_ref = orc.tridiag_eigvals(a, b)[0]
    info = ham.lanczos(max_iter=100, seed=1, storage=torch.float64, nev=3)
    assert abs(info["evals"][0] - e_ref) <= 1e-10 * abs(e_ref)
    # the first steps of the recurrence agree with the oracle's
    assert np.abs(info["alpha"][:10] - a[:10]).max() < 1e-10
    assert np.abs(info["beta"][:10] - b[:10]).max() < 1e-10
    info32 = ham.lanczos(max_iter=100, seed=1, storage=torch.float32)
    assert abs(info32["evals"][0] - e_ref) <= 1e-6 * abs(e_ref)


def test_f32_storage_matches_f64_mid_size(orc):
    """4x6 J1-J2 (N=24, dim 2,704,156): FP32 vector storage with FP64-class
    dots against the FP64 form, and the first recurrence coefficients."""
    A = api()
    bonds, J = W.square_j1j2(4, 6)
    ham = A.Hamiltonian(A.Basis(24, 12, bonds), J)
    r64 = ham.lanczos(max_iter=200, seed=2, storage=torch.float64)
    r32 = ham.lanczos(max_iter=200, seed=2, storage=torch.float32)
    assert np.abs(r32["alpha"][:5] - r64["alpha"][:5]).max() < 1e-5
    assert np.abs(r32["beta"][:5] - r64["beta"][:5]).max() < 1e-5
    assert abs(r32["evals"][0] - r64["evals"][0]) <= 1e-6 * abs(r64["evals"][0])


def test_ground_state_vector_and_residual(orc):
    A = api()
    N = 14
    bonds = W.random_bonds(N, 24, 3)
    J = W.uniform_couplings(24, 4)
    st = orc.enumerate_states(N, 7)
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    ham = A.Hamiltonian(A.Basis(N, 7, bonds), J)
    e0, psi, info = ham.ground_state(max_iter=150, seed=3)
    assert abs(e0 - w[0]) <= 1e-10 * abs(w[0])
    p = psi.cpu().numpy()
    assert abs(np.linalg.norm(p) - 1) < 1e-12
    assert abs(abs(p @ V[:, 0]) - 1) < 1e-8
    assert info["resid"][0] < 1e-6


@pytest.mark.parametrize("storage", [torch.float64, torch.float32])
def test_ground_state_two_passes_agree_on_small_blocks(orc, storage):
    """Small U(1) blocks run the first Lanczos pass in one cooperative launch
    and the second pass (the eigenvector from the recorded alpha and beta) as
    separate products; the second pass must rebuild the first pass's vectors,
    so after 250 steps (far past convergence, where a mismatch grows) the
    vector is still the ground state, in both storage types."""
    A = api()
    N = 14
    bonds, J = W.chain_j1j2(N, 1.0, 0.3)  # a single ground state (J2 = 1/2 has two)
    st = orc.enumerate_states(N, 7)
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    assert w[1] - w[0] > 1e-3
    ham = A.Hamiltonian(A.Basis(N, 7, bonds), J)
    e0, psi, info = ham.ground_state(max_iter=250, seed=5, storage=storage)
    tol = 1e-10 if storage == torch.float64 else 1e-6
    assert abs(e0 - w[0]) <= tol * abs(w[0])
    p = psi.double().cpu().numpy()
    assert abs(abs(p @ V[:, 0]) / np.linalg.norm(p) - 1) < (1e-8 if storage == torch.float64 else 1e-4)


def test_bilinear_matches_oracle(orc):
    A = api()
    # bond counts cover one to eight bonds per warp and two launches of 256
    # bonds; dimensions span one to many row tiles of 1024
    for N, nup, nb, seed in [(10, 5, 20, 1), (13, 6, 26, 2), (16, 8, 32, 3), (18, 9, 100, 4),
                             (14, 7, 91, 6), (24, 2, 270, 5)]:
        bonds = W.random_bonds(N, nb, seed)
        J = W.uniform_couplings(nb, seed)
        st = orc.enumerate_states(N, nup)
        ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
        g, x = orc.rng_normal(seed, 0, st.size), orc.rng_normal(seed + 9, 0, st.size)
        dJ = ham.bilinear(torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
        ref = orc.bond_forms(N, st, bonds, g, x)
        assert rel_l2(dJ, ref) <= 1e-12
        # deterministic: same call, same bits
        dJ2 = ham.bilinear(torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.array_equal(dJ, dJ2)
        # FP32 vectors: the sums run in FP64 on the float values
        g32, x32 = g.astype(np.float32), x.astype(np.float32)
        dJ32 = ham.bilinear(torch.from_numpy(g32).cuda(), torch.from_numpy(x32).cuda()).cpu().numpy()
        ref32 = orc.bond_forms(N, st, bonds, g32.astype(np.float64), x32.astype(np.float64))
        assert rel_l2(dJ32, ref32) <= 1e-12


def test_autograd_apply(orc):
    A = api()
    N, nup = 12, 6
    bonds = W.ladder(6, 2)
    J = W.uniform_couplings(24, 8)
    st = orc.enumerate_states(N, nup)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda", requires_grad=True)
    x = torch.from_numpy(orc.rng_normal(4, 0, st.size)).cuda().requires_grad_(True)
    c = torch.from_numpy(orc.rng_normal(5, 0, st.size)).cuda()
    loss = (c * A.heisenberg_apply(ham, Jt, x)).sum()
    loss.backward()
    ref_J = orc.bond_forms(N, st, bonds, c.cpu().numpy(), x.detach().cpu().numpy())
    ref_x = orc.apply_u1(N, st, bonds, J, c.cpu().numpy())
    assert rel_l2(Jt.grad.cpu().numpy(), ref_J) <= 1e-12
    assert rel_l2(x.grad.cpu().numpy(), ref_x) <= 1e-12


def test_energy_gradient_ladder(orc):
    """C3 pattern at oracle size: ladder with duplicated rungs, dE0/dJ by the
    backward kernel vs central finite differences and Hellmann-Feynman."""
    A = api()
    L = 6
    bonds = W.ladder(L, 2)
    N = 2 * L
    J = W.uniform_couplings(bonds.shape[0], 3)
    st = orc.enumerate_states(N, L)
    ham = A.Hamiltonian(A.Basis(N, L, bonds), J)
    Jt = torch.tensor(J, dtype=torch.float64, device="cuda", requires_grad=True)
    E = A.ground_energy(ham, Jt, max_iter=200, seed=3)
    E.backward()
    g = Jt.grad.cpu().numpy()
    w, V = np.linalg.eigh(orc.dense_u1(N, st, bonds, J))
    hf = orc.bond_forms(N, st, bonds, V[:, 0], V[:, 0])
    assert abs(E.item() - w[0]) < 1e-10 * abs(w[0])
    assert np.abs(g - hf).max() < 1e-8
    h = 1e-5
    for b in (0, 3, 2 * L, 3 * L):
        e = np.zeros_like(J); e[b] = h
        fd = (np.linalg.eigvalsh(orc.dense_u1(N, st, bonds, J + e))[0]
              - np.linalg.eigvalsh(orc.dense_u1(N, st, bonds, J - e))[0]) / (2 * h)
        assert abs(fd - g[b]) < 1e-6
    assert abs(J @ g - w[0]) < 1e-9
    assert np.abs(g[2 * L:3 * L] - g[3 * L:]).max() < 1e-9


def test_bilinear_columns_and_autograd_block(orc):
    """xd_apply_bilinear_nvec: the per-bond forms summed over the columns of
    [dim][nvec] g and x equal the sum of the single-column forms (FP64 and
    FP32; a small block and one on the FP32 batched layout), and the backward
    of a product on a block of vectors gives that sum."""
    A = api()
    for N, nup, bonds, J in [(14, 7, W.ladder(7, 2), W.uniform_couplings(28, 5)),
                             (24, 12, W.random_bonds(24, 40, 6), W.uniform_couplings(40, 6))]:
        ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            for nvec in (2, 4, 8):
                g = torch.stack([A.random_vector(ham.dim, 10 + k, dt) for k in range(nvec)], 1).contiguous()
                x = torch.stack([A.random_vector(ham.dim, 30 + k, dt) for k in range(nvec)], 1).contiguous()
                got = ham.bilinear(g, x).cpu().numpy()
                want = sum(ham.bilinear(g[:, k].contiguous(), x[:, k].contiguous()).cpu().numpy()
                           for k in range(nvec))
                assert np.abs(got - want).max() <= tol * np.abs(want).max()
    ham = A.Hamiltonian(A.Basis(14, 7, W.ladder(7, 2)), W.uniform_couplings(28, 5))
    Jt = torch.tensor(ham.J, requires_grad=True)
    x = torch.stack([A.random_vector(ham.dim, 50 + k, torch.float64) for k in range(4)], 1).contiguous()
    y = A.heisenberg_apply(ham, Jt, x)
    w = torch.stack([A.random_vector(ham.dim, 70 + k, torch.float64) for k in range(4)], 1).contiguous()
    (y * w).sum().backward()
    want = ham.bilinear(w, x).cpu().numpy()
    assert np.abs(Jt.grad.numpy() - want).max() <= 1e-12 * np.abs(want).max()


def test_basis_states_u1_and_range_errors(orc):
    """xd_basis_states on U(1) blocks: the words of a row range equal the
    oracle's enumeration (first, last and random ranges, int64 rows at N = 36
    through the counting index); ranges outside the block are XD_ERANGE."""
    A = api()
    st = orc.enumerate_states(16, 8)
    basis = A.Basis(16, 8, W.chain(16))
    assert np.array_equal(basis.states().cpu().numpy().astype(np.uint64), st)
    assert np.array_equal(basis.states(100, 37).cpu().numpy().astype(np.uint64), st[100:137])
    big = A.Basis(36, 18, W.chain(36))
    for first in (0, big.dim - 5, 2**32 - 2, 123456789):
        w = big.states(first, 5).cpu().numpy()
        assert [int(v) for v in w] == [orc.state_count(36, 18, first + k) for k in range(5)]
    from paper_2505_02901_gb300._lib import XD_ERANGE, XDError
    with pytest.raises(XDError) as e:
        basis.states(basis.dim - 2, 5)
    assert e.value.status == XD_ERANGE

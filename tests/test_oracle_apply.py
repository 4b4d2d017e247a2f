"""Pins of the oracle's H x on U(1) blocks (Eq. 1, App. A SdotS)."""
import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W
from tests._kron import heisenberg_sector


@pytest.mark.parametrize("N,nb,seed", [(2, 1, 0), (4, 5, 1), (6, 9, 2), (8, 14, 3), (10, 20, 4)])
def test_matrix_equals_kronecker_construction(orc, N, nb, seed):
    bonds = W.random_bonds(N, min(nb, N * (N - 1) // 2), seed)
    J = W.uniform_couplings(bonds.shape[0], seed + 100, -1.0, 2.0)
    for nup in range(N + 1):
        st = orc.enumerate_states(N, nup)
        Hk, idx = heisenberg_sector(N, nup, bonds, J)
        assert idx.tolist() == st.tolist()
        Ho = orc.dense_u1(N, st, bonds, J)
        assert np.abs(Ho - Hk.toarray()).max() < 1e-13


def test_two_site_singlet_energy(orc):
    st = orc.enumerate_states(2, 1)
    H = orc.dense_u1(2, st, W.chain(2), [1.0])
    assert np.allclose(np.linalg.eigvalsh(H), [-0.75, 0.25], atol=1e-15)


def test_four_site_ring(orc):
    st = orc.enumerate_states(4, 2)
    H = orc.dense_u1(4, st, W.chain(4), np.ones(4))
    assert abs(np.linalg.eigvalsh(H)[0] + 2.0) < 1e-14


def test_all_up_state_energy(orc):
    bonds = W.random_bonds(9, 15, 7)
    J = W.uniform_couplings(15, 8)
    st = orc.enumerate_states(9, 9)
    H = orc.dense_u1(9, st, bonds, J)
    assert H.shape == (1, 1) and abs(H[0, 0] - J.sum() / 4) < 1e-14


def test_hermitian_and_su2_multiplets(orc):
    N = 8
    bonds = W.random_bonds(N, 14, 11)
    J = W.uniform_couplings(14, 12)
    spectra = {}
    for nup in range(N // 2, N + 1):
        st = orc.enumerate_states(N, nup)
        H = orc.dense_u1(N, st, bonds, J)
        assert np.abs(H - H.T).max() < 1e-15
        spectra[nup] = np.linalg.eigvalsh(H)
    # [H, S^2] = 0: every level of Sz = m+1 reappears at Sz = m.
    for nup in range(N // 2, N):
        hi, lo = spectra[nup + 1], spectra[nup]
        for e in hi:
            assert np.abs(lo - e).min() < 1e-10
        assert lo[0] <= hi[0] + 1e-12


def test_symmetric_bilinear_form(orc):
    N, nup = 12, 6
    bonds = W.random_bonds(N, 20, 5)
    J = W.uniform_couplings(20, 6)
    st = orc.enumerate_states(N, nup)
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, st.size))
    Hu, Hv = orc.apply_u1(N, st, bonds, J, u), orc.apply_u1(N, st, bonds, J, v)
    assert abs(u @ Hv - Hu @ v) < 1e-11 * np.abs(u @ Hv)


def test_multi_vector_apply_is_columnwise(orc):
    N, nup = 10, 5
    bonds, J = W.chain(N), W.uniform_couplings(N, 3)
    st = orc.enumerate_states(N, nup)
    X = np.random.default_rng(1).standard_normal((st.size, 8))
    Y = orc.apply_u1(N, st, bonds, J, X)
    for v in range(8):
        assert np.abs(Y[:, v] - orc.apply_u1(N, st, bonds, J, X[:, v].copy())).max() < 1e-14


@pytest.mark.parametrize("N,nup", [(14, 7), (16, 8), (15, 4)])
def test_sampled_rows_equal_full_product(orc, N, nup):
    bonds = W.random_bonds(N, 2 * N, N)
    J = W.uniform_couplings(bonds.shape[0], N)
    st = orc.enumerate_states(N, nup)
    seed = 1234 + N
    x = orc.rng_normal(seed, 0, st.size)
    y = orc.apply_u1(N, st, bonds, J, x)
    rows = np.random.default_rng(2).integers(0, st.size, 300)
    assert np.abs(orc.apply_rows_rng(N, nup, bonds, J, seed, rows) - y[rows]).max() < 1e-13
    flips = orc.flip_index_rows(N, nup, bonds, rows)
    for k, r in enumerate(rows):
        s = int(st[r])
        for b, (i, j) in enumerate(bonds):
            if ((s >> i) & 1) == ((s >> j) & 1):
                assert flips[k, b] == -1
            else:
                assert st[flips[k, b]] == s ^ (1 << int(i)) ^ (1 << int(j))


def test_chain16_ground_energy_against_kronecker(orc):
    """C1 workload: the periodic N=16 chain at Sz=0 (dim 12870)."""
    import scipy.sparse.linalg as sla
    N = 16
    bonds = W.chain(N)
    Hk, _ = heisenberg_sector(N, 8, bonds, np.ones(N))
    e_ref = sla.eigsh(Hk, k=1, which="SA", tol=1e-14)[0][0]
    st = orc.enumerate_states(N, 8)
    v0 = orc.rng_normal(1, 0, st.size)
    alpha, beta = orc.lanczos(lambda v: orc.apply_u1(N, st, bonds, np.ones(N), v), st.size, v0, 100)
    e0 = orc.tridiag_eigvals(alpha, beta)[0]
    assert abs(e0 - e_ref) < 1e-10 * abs(e_ref)
    # thermodynamic-limit sanity: E0/N approaches 1/4 - ln 2 from below
    assert -0.4463 > e0 / N > -0.4500

"""GPU parity of the U(1) product against the oracle (a1-a5), through the C ABI."""
import math

import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu

# (N, nup, bonds, J) small enough for the full oracle; several prefix blocks
# (N > 8) and ragged block sizes (nup != N/2)
def _cases():
    out = []
    for N, nup, seed in [(2, 1, 0), (3, 1, 1), (5, 2, 2), (8, 4, 3), (9, 2, 4), (10, 5, 5),
                         (12, 6, 6), (13, 4, 7), (14, 7, 8), (16, 8, 9), (16, 3, 10), (17, 8, 11)]:
        nb = min(N * (N - 1) // 2, 2 * N)
        bonds = W.random_bonds(N, nb, seed)
        J = W.uniform_couplings(nb, seed + 50, -0.5, 1.5)
        out.append((N, nup, bonds, J))
    out.append((16, 8, W.chain(16), np.ones(16)))
    b, J = W.square_j1j2(4, 4)
    out.append((16, 8, b, J))
    out.append((20, 10, W.ladder(10, 2), W.uniform_couplings(40, 3)))
    # block-structured path (N >= 20): irregular graphs mixing prefix,
    # postfix and cross bonds, ragged block sizes (nup != N/2)
    out.append((21, 7, W.random_bonds(21, 42, 21), W.uniform_couplings(42, 21, -1.0, 1.0)))
    out.append((22, 11, W.random_bonds(22, 60, 22), W.uniform_couplings(60, 22)))
    b, J = W.square_j1j2(4, 6)
    out.append((24, 12, b, J))
    out.append((24, 9, W.random_bonds(24, 30, 24), W.uniform_couplings(30, 24)))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_apply_f64_matches_oracle(orc, case):
    A = api()
    N, nup, bonds, J = CASES[case]
    st = orc.enumerate_states(N, nup)
    basis = A.Basis(N, nup, bonds)
    assert basis.dim == st.size == math.comb(N, nup)
    ham = A.Hamiltonian(basis, J)
    x = orc.rng_normal(100 + case, 0, st.size)
    y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert rel_l2(y, yo) <= 1e-12
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("case", [3, 6, 9, 12, 13, 14, 16, 17, 18])
@pytest.mark.parametrize("nvec", [1, 2, 4, 8])
def test_apply_f32_and_multi_rhs(orc, case, nvec):
    A = api()
    N, nup, bonds, J = CASES[case]
    st = orc.enumerate_states(N, nup)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    X = np.stack([orc.rng_normal(7 + k, 0, st.size) for k in range(nvec)], axis=1)
    Yo = orc.apply_u1(N, st, bonds, J, X)
    x32 = torch.from_numpy(X.astype(np.float32)).cuda().contiguous()
    y32 = ham.apply(x32 if nvec > 1 else x32[:, 0].contiguous()).cpu().numpy().reshape(st.size, nvec)
    # float storage: inputs rounded to float, float accumulation of <= 2N terms
    Yo32 = orc.apply_u1(N, st, bonds, J, X.astype(np.float32).astype(np.float64))
    assert rel_l2(y32, Yo32) <= 2e-6
    assert rel_l2(y32, Yo) <= 4e-6
    if nvec > 1:
        y64 = ham.apply(torch.from_numpy(X).cuda().contiguous()).cpu().numpy()
        assert rel_l2(y64, Yo) <= 1e-12


def test_index_maps_bit_exact(orc):
    A = api()
    for N, nup in [(12, 6), (16, 8), (17, 5), (28, 14), (32, 16), (36, 18)]:
        basis = A.Basis(N, nup, W.chain(N))
        assert basis.dim == math.comb(N, nup)
        rng = np.random.default_rng(N)
        idx = np.concatenate([[0, basis.dim - 1], rng.integers(0, basis.dim, 200)])
        for k in idx:
            s = basis.state(int(k))
            assert s == orc.state_count(N, nup, int(k))
            assert basis.index(s) == k
        assert basis.index((1 << (nup + 1)) - 1) == -1  # wrong popcount


def test_random_vector_matches_oracle_generator(orc):
    A = api()
    for seed in (0, 1, 12345):
        x = A.random_vector(5000, seed, torch.float64).cpu().numpy()
        xo = orc.rng_normal(seed, 0, 5000)
        assert np.abs(x - xo).max() <= 1e-14 * np.abs(xo).max()
        x32 = A.random_vector(5000, seed, torch.float32).cpu().numpy()
        assert np.array_equal(x32, xo.astype(np.float32)) or np.abs(x32 - xo).max() < 1e-6


def test_edge_cases(orc):
    A = api()
    # one-state sectors: all down, all up
    for nup in (0, 10):
        bonds = W.chain(10)
        ham = A.Hamiltonian(A.Basis(10, nup, bonds), np.ones(10))
        y = ham.apply(torch.ones(1, dtype=torch.float64, device="cuda")).cpu().numpy()
        assert abs(y[0] - 10 / 4) < 1e-15
    # two sites, one bond: eigenvalues -3/4 (singlet), 1/4
    ham = A.Hamiltonian(A.Basis(2, 1, W.chain(2)), [1.0])
    H = np.stack([ham.apply(torch.tensor(e, device="cuda")).cpu().numpy()
                  for e in np.eye(2)], axis=1)
    assert np.allclose(np.linalg.eigvalsh(H), [-0.75, 0.25], atol=1e-15)


def test_errors_are_statuses(orc):
    A = api()
    from paper_2505_02901_gb300._lib import XD_EINVAL, XD_ERANGE, XDError
    with pytest.raises(XDError) as e:
        A.Basis(8, 4, [[0, 0]])
    assert e.value.status == XD_EINVAL
    with pytest.raises(XDError) as e:
        A.Basis(8, 4, [[0, 8]])
    assert e.value.status == XD_EINVAL
    with pytest.raises(XDError) as e:
        A.Basis(41, 2, [[0, 1]])
    assert e.value.status == XD_ERANGE
    with pytest.raises(XDError) as e:
        A.Basis(8, 9, [[0, 1]])
    assert e.value.status == XD_EINVAL
    ham = A.Hamiltonian(A.Basis(8, 4, W.chain(8)), np.ones(8))
    x = torch.zeros(70, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(XDError) as e:
        ham.apply(x)  # nvec = 3
    assert e.value.status == XD_EINVAL
    with pytest.raises(XDError):
        ham.apply(torch.zeros(70, dtype=torch.complex128, device="cuda"))
    with pytest.raises(XDError):
        A.Hamiltonian(A.Basis(8, 4, W.chain(8)), [1, 2, 3, 4, 5, 6, 7, float("nan")])


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
def test_ladder28_full_size(orc, dtype, tol):
    """C3 workload size: 14x2 ladder, 56 bonds (each rung twice), dim
    40,116,600; sampled rows against the counting-index oracle."""
    A = api()
    bonds = W.ladder(14, 2)
    J = W.uniform_couplings(56, 3)
    ham = A.Hamiltonian(A.Basis(28, 14, bonds), J)
    assert ham.dim == 40116600
    seed = 77
    x = A.random_vector(ham.dim, seed, dtype)
    y = ham.apply(x)
    rows = np.concatenate([[0, ham.dim - 1], np.random.default_rng(1).integers(0, ham.dim, 3000)])
    yo = orc.apply_rows_rng(28, 14, bonds, J, seed, rows)
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert rel_l2(ys, yo) <= tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 5e-6)])
def test_square4x8_full_size(orc, dtype, tol):
    """C2 workload: 4x8 J1-J2 (J1=1, J2=0.5), N=32, Sz=0, dim 601,080,390."""
    A = api()
    bonds, J = W.square_j1j2(4, 8)
    ham = A.Hamiltonian(A.Basis(32, 16, bonds), J)
    assert ham.dim == 601080390
    seed = 2
    x = A.random_vector(ham.dim, seed, dtype)
    y = ham.apply(x)
    rows = np.concatenate([[0, ham.dim - 1, ham.dim // 2],
                           np.random.default_rng(2).integers(0, ham.dim, 2000)])
    yo = orc.apply_rows_rng(32, 16, bonds, J, seed, rows)
    ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert rel_l2(ys, yo) <= tol
    del x, y
    torch.cuda.empty_cache()


def test_eight_rhs_large_block(orc):
    """Eight FP32 right-hand sides on a ragged N=26 block with prefix, postfix
    and cross bonds (the eight-vector form of the batched layout), and the
    same product from a vector that is not 16-byte aligned (generic kernel)."""
    A = api()
    N, nup = 26, 12
    bonds, J = W.random_bonds(N, 52, 26), W.uniform_couplings(52, 26, -1.0, 1.0)
    st = orc.enumerate_states(N, nup)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    X = np.stack([orc.rng_normal(30 + k, 0, st.size) for k in range(8)], axis=1).astype(np.float32)
    Yo = orc.apply_u1(N, st, bonds, J, X.astype(np.float64))
    x = torch.from_numpy(X).cuda().contiguous()
    y = ham.apply(x).cpu().numpy()
    assert rel_l2(y, Yo) <= 2e-6
    buf = torch.empty(st.size * 8 + 1, dtype=torch.float32, device="cuda")
    xu = buf[1:].view(st.size, 8)
    xu.copy_(x)
    yu = ham.apply(xu).cpu().numpy()
    assert rel_l2(yu, Yo) <= 2e-6

"""GPU parity of the FP64 product on large U(1) blocks (N >= 24), which runs in
double-float arithmetic on the FP32 pipe with one FP64 addition per row,
against the FP64 oracle at the FP64 tolerance (relative L2 <= 1e-12), and
its handling of vectors of any magnitude (the power-of-two scaling of the
split), zeros, subnormal entries and non-finite entries."""
import math

import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def _cases():
    out = []
    b, J = W.square_j1j2(4, 6)
    out.append(("square4x6", 24, 12, b, J))
    # random graphs: prefix, postfix and cross bonds of every kind, ragged
    # classes (nup != N/2), couplings that are not exact in FP32
    out.append(("random24_9", 24, 9, W.random_bonds(24, 60, 31), W.uniform_couplings(60, 31, -1.0, 1.5)))
    out.append(("random25_12", 25, 12, W.random_bonds(25, 70, 32), W.uniform_couplings(70, 32, -0.7, 1.3)))
    out.append(("random26_13", 26, 13, W.random_bonds(26, 52, 33), W.uniform_couplings(52, 33)))
    out.append(("random26_7", 26, 7, W.random_bonds(26, 80, 34), W.uniform_couplings(80, 34, -2.0, 2.0)))
    out.append(("ladder26", 26, 13, W.ladder(13, 2), W.uniform_couplings(52, 35)))
    out.append(("chain27_11", 27, 11, W.chain(27), np.full(27, 1.0 / 3.0)))
    return out


CASES = _cases()


@pytest.fixture(scope="module")
def blocks(orc):
    cache = {}

    def get(k):
        if k not in cache:
            name, N, nup, bonds, J = CASES[k]
            A = api()
            ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
            cache.clear()
            cache[k] = (ham, orc.enumerate_states(N, nup))
        return cache[k]
    return get


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
def test_f64_product_matches_oracle(orc, blocks, case):
    name, N, nup, bonds, J = CASES[case]
    ham, st = blocks(case)
    assert ham.dim == st.size == math.comb(N, nup)
    x = orc.rng_normal(200 + case, 0, st.size)
    y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert rel_l2(y, yo) <= 1e-12
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("scale", [1e-300, 1e-200, 1e-30, 1.0, 1e30, 1e200, 1e300])
def test_f64_product_at_any_magnitude(orc, blocks, scale):
    # the split scales x by a power of two chosen from its largest entry, so
    # the FP32 pairs stay in range for vectors of any magnitude
    name, N, nup, bonds, J = CASES[1]
    ham, st = blocks(1)
    x = orc.rng_normal(7, 0, st.size) * scale
    y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert np.all(np.isfinite(y))
    # compared after dividing by the scale (numpy's norm of a 1e300 vector overflows)
    assert rel_l2(y / scale, yo / scale) <= 1e-12


def test_f64_product_wide_dynamic_range_and_zeros(orc, blocks):
    # entries spread over 60 decades, a third of them exactly zero; entries
    # far below the largest lose only what the FP64 tolerance allows
    name, N, nup, bonds, J = CASES[0]
    ham, st = blocks(0)
    rng = np.random.default_rng(5)
    x = orc.rng_normal(9, 0, st.size) * 10.0 ** rng.uniform(-30, 30, st.size)
    x[rng.random(st.size) < 1 / 3] = 0.0
    y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert rel_l2(y, yo) <= 1e-12
    # the zero vector gives exactly zero
    z = ham.apply(torch.zeros(st.size, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.all(z == 0.0)
    # a unit vector: one column of H, exactly representable entries
    e = np.zeros(st.size)
    e[12345] = 1.0
    ye = ham.apply(torch.from_numpy(e).cuda()).cpu().numpy()
    yeo = orc.apply_u1(N, st, bonds, J, e)
    assert rel_l2(ye, yeo) <= 1e-14


def test_f64_product_subnormal_and_nonfinite_entries(orc, blocks):
    name, N, nup, bonds, J = CASES[0]
    ham, st = blocks(0)
    x = orc.rng_normal(11, 0, st.size)
    x[::1000] = 5e-324  # subnormal doubles: taken as zero, far below the tolerance
    y = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_l2(y, orc.apply_u1(N, st, bonds, J, x)) <= 1e-12
    # a non-finite entry makes every entry of y NaN (documented behaviour)
    for bad in (np.nan, np.inf):
        xb = x.copy()
        xb[777] = bad
        yb = ham.apply(torch.from_numpy(xb).cuda()).cpu().numpy()
        assert np.all(np.isnan(yb))
    # and the next finite product is unaffected
    y2 = ham.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y, y2)


def test_f64_product_deterministic_and_lanczos(orc, blocks):
    name, N, nup, bonds, J = CASES[0]
    ham, st = blocks(0)
    x = torch.from_numpy(orc.rng_normal(3, 0, st.size)).cuda()
    y1 = ham.apply(x)
    y2 = ham.apply(x)
    assert torch.equal(y1, y2)
    # FP64 Lanczos on the 4x6 J1-J2 lattice through this product against the
    # oracle's plain three-term Lanczos from the same start
    info = ham.lanczos(max_iter=80, seed=4)
    ref = orc.lanczos(lambda v: orc.apply_u1(N, st, bonds, J, v), st.size, orc.rng_normal(4, 0, st.size), 80,
                      full_reorth=False)
    k = min(10, info["n_iter"])
    assert np.allclose(info["alpha"][:k], ref[0][:k], rtol=0, atol=1e-10)
    e0 = float(info["evals"][0])
    e0o = float(orc.tridiag_eigvals(ref[0], ref[1])[0])
    assert abs(e0 - e0o) <= 1e-10 * abs(e0o)


def test_f64_full_size_spiky_vector_keeps_the_tolerance(orc):
    """4x8 J1-J2 (dim 601,080,390; couplings with a quantum, so fixed point is
    allowed): x = seeded normal vector + c e_0 with c = 3e4.  Rounded to the
    fixed-point grid of its largest entry, the normal part would lose about
    sqrt(dim) 2^-52 c / |x| ~ 5e-12 relative; the device's choice must take
    double-float here.  Expected rows by linearity: the oracle's rows of H x_rng
    plus c times column 0 of H (the diagonal of state 0 and J/2 at the states
    its bonds flip to, by the counting index)."""
    A = api()
    N, nup = 32, 16
    bonds, J = W.square_j1j2(4, 8)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    seed, c = 2, 3e4
    x = A.random_vector(ham.dim, seed, torch.float64)
    x[0] += c
    y = ham.apply(x)
    s0 = orc.state_count(N, nup, 0)
    pairs = [(int(i), int(j)) for i, j in bonds]  # Python ints: 1 << 31 must not wrap
    col = {0: sum(0.25 * J[b] * (1 if ((s0 >> i) & 1) == ((s0 >> j) & 1) else -1)
                  for b, (i, j) in enumerate(pairs))}
    for b, (i, j) in enumerate(pairs):
        if ((s0 >> i) & 1) != ((s0 >> j) & 1):
            r = orc.index_count(N, nup, s0 ^ (1 << i) ^ (1 << j))
            col[r] = col.get(r, 0.0) + 0.5 * J[b]
    rows = np.concatenate([np.array(sorted(col), dtype=np.int64),
                           np.random.default_rng(4).integers(0, ham.dim, 2000)])
    yo = orc.apply_rows_rng(N, nup, bonds, J, seed, rows) + c * np.array([col.get(int(r), 0.0) for r in rows])
    ys = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    # the sampled random rows alone (the spike's column is far larger)
    k = len(col)
    assert rel_l2(ys[k:], yo[k:]) <= 1e-12
    assert rel_l2(ys, yo) <= 1e-12
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nb", [300, 400])
def test_f64_dense_random_graphs_n32(orc, nb):
    """Random graphs on N = 32 (dim 601,080,390): with 300 bonds the prefix
    bonds need four 12-bit windows (four passes); with 400 bonds four windows
    cannot hold them and the FP64 product falls back to the FP64 block
    kernel.  Both meet the tolerance on sampled rows."""
    A = api()
    N, nup = 32, 16
    bonds = W.random_bonds(N, nb, 5)
    J = W.uniform_couplings(nb, 5)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    seed = 8
    x = A.random_vector(ham.dim, seed, torch.float64)
    y = ham.apply(x)
    del x
    rows = np.concatenate([[0, ham.dim - 1], np.random.default_rng(8).integers(0, ham.dim, 1000)])
    yo = orc.apply_rows_rng(N, nup, bonds, J, seed, rows)
    assert rel_l2(y[torch.from_numpy(rows).cuda()].cpu().numpy(), yo) <= 1e-12
    del y
    torch.cuda.empty_cache()

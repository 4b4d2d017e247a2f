"""Pins of the oracle's finite-temperature Lanczos thermodynamics."""
import numpy as np

from paper_2505_02901_gb300 import workloads as W


def _exact(w, temps):
    out = []
    for T in temps:
        p = np.exp(-(w - w.min()) / T)
        z = p.sum()
        E = (w * p).sum() / z
        out.append((z * np.exp(-w.min() / T), E, ((w * w * p).sum() / z - E * E) / T ** 2))
    return out


def test_orthonormal_starts_give_the_exact_trace(orc):
    """With the unit vectors e_k of the block as starts and enough steps, the
    Lanczos quadrature reproduces Tr e^{-H/T} exactly: Z, E, C equal the full
    diagonalisation at every temperature."""
    N = 8
    st = orc.enumerate_states(N, 4)
    bonds, J = W.random_bonds(N, 12, 3), W.uniform_couplings(12, 3)
    H = orc.dense_u1(N, st, bonds, J)
    mv = lambda v: H @ v  # noqa: E731
    starts = list(np.eye(st.size))
    tri = orc.ftlm_tridiagonals(mv, starts, st.size)
    temps = [0.1, 0.5, 1.0, 4.0]
    got = orc.ftlm_thermo(tri, st.size, temps, exact_trace=True)
    ref = _exact(np.linalg.eigvalsh(H), temps)
    for (z, e, c), (z0, e0, c0) in zip(got, ref):
        assert abs(z / z0 - 1) < 1e-9 and abs(e - e0) < 1e-9 and abs(c - c0) < 1e-8


def test_random_starts_high_temperature_and_ground_state(orc):
    """Random starts: at T -> infinity E approaches Tr H / dim (each estimate
    is unbiased); at low T it approaches E0."""
    N = 12
    st = orc.enumerate_states(N, 6)
    H = orc.dense_u1(N, st, W.chain(N), np.ones(N))
    w = np.linalg.eigvalsh(H)
    starts = [orc.rng_normal(100 + r, 0, st.size) for r in range(32)]
    tri = orc.ftlm_tridiagonals(lambda v: H @ v, starts, 60)
    (_, e_hi, _), (_, e_lo, _) = orc.ftlm_thermo(tri, st.size, [1e4, 0.02])
    assert abs(e_hi - w.mean()) < 0.05 * np.abs(w).max()
    assert abs(e_lo - w[0]) < 1e-6


def test_lanczos_on_a_complex_block(orc):
    """The oracle's Lanczos on a complex (momentum 2 pi / 12) block of the
    chain: Hermitian inner products, real tridiagonal, its extreme Ritz
    values equal to numpy's eigenvalues of the dense block."""
    from paper_2505_02901_gb300 import workloads as W
    blk = orc.SymBlock(12, 6, W.chain_translations(12), W.chain_characters(12, 1))
    H = blk.dense(W.chain(12), np.ones(12))
    assert np.abs(H.imag).max() > 1e-3 and np.abs(H - H.conj().T).max() < 1e-14
    a, b = orc.lanczos(lambda v: H @ v, blk.dim, orc.rng_normal(3, 0, blk.dim).astype(complex), 60)
    assert a.dtype == np.float64 and b.dtype == np.float64
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    w, wt = np.linalg.eigvalsh(H), np.sort(np.linalg.eigvalsh(T))
    assert np.abs(wt[:3] - w[:3]).max() < 1e-12 and abs(wt[-1] - w[-1]) < 1e-12

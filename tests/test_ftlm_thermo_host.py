"""The library's host thermodynamics of finite-temperature Lanczos
(xd_ftlm_thermo, no GPU needed) against the oracle on the same tridiagonals."""
import numpy as np

from paper_2505_02901_gb300 import workloads as W


def test_thermo_matches_oracle(orc):
    from paper_2505_02901_gb300 import api as A
    N = 10
    st = orc.enumerate_states(N, 5)
    H = orc.dense_u1(N, st, W.chain(N), np.ones(N))
    R, M = 6, 30
    tri = orc.ftlm_tridiagonals(lambda v: H @ v, [orc.rng_normal(9 + r, 0, st.size) for r in range(R)], M)
    a = np.array([t[0] for t in tri])
    b = np.array([t[1] for t in tri])
    n = np.full(R, M, dtype=np.int32)
    temps = [0.05, 0.3, 1.0, 10.0]
    Z, E, C = A.ftlm_thermo(a, b, n, st.size, temps)
    ref = orc.ftlm_thermo(tri, st.size, temps)
    for q, (z0, e0, c0) in enumerate(ref):
        assert abs(Z[q] / z0 - 1) < 1e-10 and abs(E[q] - e0) < 1e-10 and abs(C[q] - c0) < 1e-8

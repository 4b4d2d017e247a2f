"""Independent construction of the Heisenberg matrix for small N.

H = sum_b J_b (Sx_i Sx_j + Sy_i Sy_j + Sz_i Sz_j) built from Kronecker
products of the spin-1/2 matrices S = sigma/2 on the full 2^N space
(Eq. 1 and the SdotS type of App. A), then restricted to the words with nup
set bits.  Basis word w has site i in bit i (1 = up), so site i is the
(N-1-i)-th Kronecker factor from the left.  Shares nothing with the oracle.
"""
import numpy as np
import scipy.sparse as sp

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128) / 2
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128) / 2
# |0> = down (bit 0), |1> = up (bit 1): Sz = diag(-1/2, +1/2)
SZ = np.array([[-1, 0], [0, 1]], dtype=np.complex128) / 2


def _site_op(op, i, N):
    mats = [sp.identity(2, format="csr", dtype=np.complex128)] * N
    mats = list(mats)
    mats[N - 1 - i] = sp.csr_matrix(op)
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out


def heisenberg_full(N, bonds, J):
    dim = 2 ** N
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    cache = {}

    def op(o, i):
        key = (id(o), i)
        if key not in cache:
            cache[key] = _site_op(o, i, N)
        return cache[key]

    for (i, j), c in zip(bonds, J):
        for o in (SX, SY, SZ):
            H = H + c * (op(o, int(i)) @ op(o, int(j)))
    return H


def heisenberg_sector(N, nup, bonds, J):
    H = heisenberg_full(N, bonds, J)
    idx = np.array([w for w in range(2 ** N) if bin(w).count("1") == nup], dtype=np.int64)
    Hs = H[idx][:, idx]
    assert abs(Hs.imag).max() < 1e-14 if Hs.nnz else True
    return Hs.real.tocsr(), idx

"""Host-side validation of xd_basis_create, which runs before any CUDA call
and therefore runs here without a GPU: every malformed block or group comes
back as a status with a message, and no handle is returned."""
import ctypes

import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W


@pytest.fixture(scope="module")
def L():
    from paper_2505_02901_gb300 import _lib
    return _lib


def _create(L, N, nup, bonds, perms=None, chi=None, ngroup=None):
    lib = L.lib()
    b = None if bonds is None else np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    bp = None if b is None else b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    nb = 0 if b is None else b.shape[0]
    sym_p, keep = None, []
    if perms is not None:
        p = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
        c = np.asarray(chi, dtype=np.complex128)
        cr, ci = np.ascontiguousarray(c.real), np.ascontiguousarray(c.imag)
        keep = [p, cr, ci]
        sym = L.xd_symmetry(p.shape[0] if ngroup is None else ngroup,
                            p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            cr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            ci.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        sym_p = ctypes.byref(sym)
    out = ctypes.c_void_p(12345)
    st = lib.xd_basis_create(N, nup, bp, nb, sym_p, ctypes.byref(out))
    del keep
    return st, out.value, lib.xd_last_error().decode()


def _rejects(L, status, word, *args, **kw):
    st, h, msg = _create(L, *args, **kw)
    assert st == status, (st, msg)
    assert h is None  # *out is cleared on failure
    assert word in msg, msg


def test_block_arguments(L):
    ch = W.chain(8)
    _rejects(L, L.XD_EINVAL, "N", 1, 0, [(0, 0)])
    _rejects(L, L.XD_ERANGE, "N", 41, 20, W.chain(41))
    _rejects(L, L.XD_EINVAL, "nup", 8, -1, ch)
    _rejects(L, L.XD_EINVAL, "nup", 8, 9, ch)
    _rejects(L, L.XD_EINVAL, "bonds", 8, 4, None)
    _rejects(L, L.XD_ERANGE, "bonds", 8, 4, np.tile(ch, (513, 1)))  # 4104 bonds
    _rejects(L, L.XD_EINVAL, "invalid", 8, 4, [(0, 1), (2, 2)])
    _rejects(L, L.XD_EINVAL, "invalid", 8, 4, [(0, 1), (3, 8)])
    _rejects(L, L.XD_EINVAL, "invalid", 8, 4, [(0, 1), (-1, 3)])


def test_group_size_and_arrays(L):
    ch, T = W.chain(8), W.chain_translations(8)
    chi = W.chain_characters(8, 0)
    _rejects(L, L.XD_EINVAL, "ngroup", 8, 4, ch, T, chi, ngroup=0)
    big = np.tile(T, (257, 1))  # 2056 rows
    _rejects(L, L.XD_EINVAL, "ngroup", 8, 4, ch, big, np.ones(len(big)))


def test_group_axioms(L):
    N = 8
    ch, T = W.chain(N), W.chain_translations(N)
    chi = W.chain_characters(N, 1)
    bad = T.copy()
    bad[3, 0] = bad[3, 1]  # not a permutation
    _rejects(L, L.XD_ESYM, "permutation", N, 4, ch, bad, chi)
    dup = np.vstack([T, T[2:3]])  # an element listed twice
    _rejects(L, L.XD_ESYM, "more than once", N, 4, ch, dup, np.r_[chi, chi[2:3]])
    _rejects(L, L.XD_ESYM, "identity", N, 4, ch, T[1:], chi[1:])  # identity missing
    _rejects(L, L.XD_ESYM, "closed", N, 4, ch, T[:5], chi[:5])  # not closed
    c2 = chi.copy()
    c2[1] *= 1.5  # |chi| != 1
    _rejects(L, L.XD_ESYM, "|chi(g)| != 1", N, 4, ch, T, c2)
    c3 = chi.copy()
    c3[2] = 1.0  # not a homomorphism
    _rejects(L, L.XD_ESYM, "homomorphism", N, 4, ch, T, c3)
    _rejects(L, L.XD_ESYM, "bond graph", N, 4, ch[:-1], T, chi)  # open chain is not invariant


def test_wide_group_checks_run_on_the_host(L):
    """The 432-element space group of the 6x6 triangular torus passes the
    group axioms on the host (hashed closure test): with characters that
    break the homomorphism the call is rejected as a symmetry error, quickly."""
    import time
    b, _ = W.triangular(6)
    g = W.space_group(6, 6, "triangular")
    c = W.space_group_characters(6, 6, "triangular").copy()
    c[len(c) // 2] = -1.0  # a mirror class made inconsistent
    t0 = time.perf_counter()
    _rejects(L, L.XD_ESYM, "homomorphism", 36, 18, b, g, c)
    assert time.perf_counter() - t0 < 30
    # a square-lattice mirror does not map the triangular bonds onto themselves
    gs = W.space_group(6, 6, "square")
    _rejects(L, L.XD_ESYM, "bond graph", 36, 18, b, gs, np.ones(len(gs)))


def test_injected_allocation_failure_is_an_out_of_memory_status(L):
    """With an allocation failure injected at the first device allocation,
    creating a valid block fails as XD_ENOMEM (on the host, before any other
    CUDA call) and returns no handle; the injection is then off again."""
    lib = L.lib()
    assert lib.xd_debug_fail_alloc(0) == L.XD_OK
    try:
        st, h, msg = _create(L, 12, 6, W.chain(12))
        assert st == L.XD_ENOMEM and h is None
        assert "allocation" in msg.lower() or "memory" in msg.lower(), msg
    finally:
        lib.xd_debug_fail_alloc(-1)

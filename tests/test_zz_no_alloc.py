"""GPU test of xd_apply_bilinear_noalloc, the bilinear-forms entry point that
allocates nothing (for callers whose own allocator owns the device memory,
or that cannot afford cudaMalloc/cudaFree inside their loop).

It is called through the C ABI (ctypes) and compared with the allocating
xd_apply_bilinear on the same inputs, twice in a row, because every call
reuses the same fixed device array.  The file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_02901_gb300 import workloads as W
from tests.gpu_common import api, rel_l2

pytestmark = pytest.mark.gpu


def _call(fn, ham, g, x, dtype_code, out):
    from paper_2505_02901_gb300 import _lib
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = fn(ham._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(x.data_ptr()), dtype_code,
                ctypes.c_void_p(out.data_ptr()), st)
    return status, _lib.lib().xd_last_error().decode()


@pytest.mark.parametrize("N,nup,nb,dtype", [(14, 7, 28, torch.float64), (20, 9, 40, torch.float64),
                                            (22, 11, 44, torch.float32)])
def test_noalloc_matches_allocating_entry_point(orc, N, nup, nb, dtype):
    A = api()
    from paper_2505_02901_gb300 import _lib
    L = _lib.lib()
    bonds = W.random_bonds(N, nb, N)
    J = W.uniform_couplings(nb, N)
    ham = A.Hamiltonian(A.Basis(N, nup, bonds), J)
    code = _lib.XD_F64 if dtype == torch.float64 else _lib.XD_F32
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    for call in range(2):
        g = A.random_vector(ham.dim, 100 + call, dtype)
        x = A.random_vector(ham.dim, 200 + call, dtype)
        ref = torch.empty(nb, dtype=torch.float64, device="cuda")
        out = torch.full((nb,), float("nan"), dtype=torch.float64, device="cuda")
        st, msg = _call(L.xd_apply_bilinear, ham, g, x, code, ref)
        assert st == _lib.XD_OK, msg
        st, msg = _call(L.xd_apply_bilinear_noalloc, ham, g, x, code, out)
        assert st == _lib.XD_OK, msg
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= tol


def test_noalloc_rejects_what_it_cannot_hold(orc):
    A = api()
    from paper_2505_02901_gb300 import _lib
    L = _lib.lib()
    N = 24
    bonds = W.random_bonds(N, 257, 1)  # one bond more than the fixed scratch holds
    ham = A.Hamiltonian(A.Basis(N, 2, bonds), np.ones(257))
    v = torch.ones(ham.dim, dtype=torch.float64, device="cuda")
    out = torch.zeros(257, dtype=torch.float64, device="cuda")
    st, msg = _call(L.xd_apply_bilinear_noalloc, ham, v, v, _lib.XD_F64, out)
    assert st == _lib.XD_ERANGE and "256" in msg
    sym = A.Basis(8, 4, W.chain(8), symmetry=(W.chain_translations(8), W.chain_characters(8, 0)))
    hs = A.Hamiltonian(sym, np.ones(8))
    v = torch.ones(sym.dim, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, msg = _call(L.xd_apply_bilinear_noalloc, hs, v, v, _lib.XD_F64, out)
    assert st == _lib.XD_EINVAL and "U(1)" in msg

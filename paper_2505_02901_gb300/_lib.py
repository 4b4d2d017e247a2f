"""ctypes binding of libxdgpu.so (argument marshalling only).

Every function of include/xdiag_gpu.h is declared here with the same name.
There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxdgpu.so")

XD_OK, XD_EINVAL, XD_ERANGE, XD_ENOMEM, XD_ECUDA, XD_ESYM, XD_ENOTCONV = range(7)
XD_F64, XD_F32, XD_C128 = 0, 1, 2
STATUS_NAMES = {0: "XD_OK", 1: "XD_EINVAL", 2: "XD_ERANGE", 3: "XD_ENOMEM", 4: "XD_ECUDA",
                5: "XD_ESYM", 6: "XD_ENOTCONV"}


class XDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class xd_symmetry(ctypes.Structure):
    _fields_ = [("ngroup", ctypes.c_int),
                ("perms", ctypes.POINTER(ctypes.c_int32)),
                ("chi_re", ctypes.POINTER(ctypes.c_double)),
                ("chi_im", ctypes.POINTER(ctypes.c_double))]


_c = ctypes
_vp, _i, _i64, _u64, _dp = _c.c_void_p, _c.c_int, _c.c_int64, _c.c_uint64, _c.POINTER(_c.c_double)
SIGNATURES = {
    "xd_basis_create": (_i, [_i, _i, _c.POINTER(_c.c_int32), _i, _c.POINTER(xd_symmetry), _c.POINTER(_vp)]),
    "xd_basis_dim": (_i, [_vp, _c.POINTER(_i64)]),
    "xd_basis_is_complex": (_i, [_vp, _c.POINTER(_i)]),
    "xd_basis_state": (_i, [_vp, _i64, _c.POINTER(_u64)]),
    "xd_basis_index": (_i, [_vp, _u64, _c.POINTER(_i64)]),
    "xd_basis_states": (_i, [_vp, _i64, _i64, _vp, _vp]),
    "xd_basis_destroy": (None, [_vp]),
    "xd_ham_create": (_i, [_vp, _dp, _c.POINTER(_vp)]),
    "xd_ham_set_couplings": (_i, [_vp, _dp]),
    "xd_ham_destroy": (None, [_vp]),
    "xd_apply": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "xd_apply_bilinear": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "xd_apply_bilinear_noalloc": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "xd_apply_bilinear_nvec": (_i, [_vp, _vp, _vp, _i, _i, _vp, _vp]),
    "xd_correlations": (_i, [_vp, _vp, _i, _c.POINTER(_c.c_int32), _i, _i, _dp]),
    "xd_evolve": (_i, [_vp, _vp, _c.c_double, _c.c_double, _i, _c.c_double, _vp, _c.POINTER(_i), _dp]),
    "xd_ftlm": (_i, [_vp, _i, _i, _u64, _dp, _dp, _c.POINTER(_i)]),
    "xd_ftlm_thermo": (_i, [_i, _i, _dp, _dp, _c.POINTER(_i), _c.c_double, _i, _dp, _dp, _dp, _dp]),
    "xd_lanczos_eigenvalues": (_i, [_vp, _i, _u64, _i, _i, _dp, _dp, _c.POINTER(_i), _dp, _dp]),
    "xd_lanczos_ground_state": (_i, [_vp, _i, _u64, _i, _i, _dp, _dp, _c.POINTER(_i), _dp, _dp, _vp]),
    "xd_energy_grad": (_i, [_vp, _vp, _i, _dp]),
    "xd_random_vector": (_i, [_i64, _u64, _vp, _i, _vp]),
    "xd_batch_apply": (_i, [_i, _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp), _i, _i, _vp]),
    "xd_last_error": (_c.c_char_p, []),
    "xd_version": (_c.c_char_p, []),
    "xd_debug_fail_alloc": (_i, [_i64]),
}

_lib = None


def lib():
    """Load libxdgpu.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                               "paper_2505_02901_gb300.build.build() (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != XD_OK:
        raise XDError(status, lib().xd_last_error().decode())

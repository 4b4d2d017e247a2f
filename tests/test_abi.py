"""The C-ABI library loads and exports every symbol of include/xdiag_gpu.h
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "xdiag_gpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(xd_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2505_02901_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), f"{n} declared in xdiag_gpu.h but not exported"


def test_binding_declares_the_same_names():
    from paper_2505_02901_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _declared()


def test_version_and_error_without_gpu():
    from paper_2505_02901_gb300 import _lib
    L = _lib.lib()
    assert b"sm_103a" in L.xd_version()
    # argument validation happens before any CUDA call
    out = ctypes.c_void_p()
    assert L.xd_basis_create(2, 1, None, 0, None, ctypes.byref(out)) == _lib.XD_EINVAL
    assert b"bonds" in L.xd_last_error()

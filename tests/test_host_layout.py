"""The library's U(1) index layout (csrc/xd_layout.h: Lin's two tables,
Sec. 3.1 and 5.2) compiled alone with g++: rank and unrank against the
oracle's enumeration (every word, N <= 16) and its counting index (sampled
words up to N = 40, int64 indices)."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_02901_gb300", "csrc")


@pytest.fixture(scope="module")
def lay():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, f"libhostlayout.{os.getpid()}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", so,
                           os.path.join(HERE, "host_layout_shim.cpp")])
    L = ctypes.CDLL(so)
    os.remove(so)
    L.shim_u1_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_int)]
    L.shim_u1_index.restype = ctypes.c_longlong
    L.shim_u1_index.argtypes = [ctypes.c_ulonglong]
    L.shim_u1_state.restype = ctypes.c_ulonglong
    L.shim_u1_state.argtypes = [ctypes.c_longlong]
    return L


def _build(lay, N, nup):
    dim, L = ctypes.c_longlong(), ctypes.c_int()
    assert lay.shim_u1_build(N, nup, ctypes.byref(dim), ctypes.byref(L)) == 1
    return dim.value, L.value


@pytest.mark.parametrize("N", [2, 5, 8, 9, 12, 16])
def test_every_word_small_blocks(lay, orc, N):
    for nup in range(N + 1):
        dim, _ = _build(lay, N, nup)
        assert dim == math.comb(N, nup)
        st = orc.enumerate_states(N, nup)
        for k, s in enumerate(st.tolist()):
            assert lay.shim_u1_index(s) == k
            assert lay.shim_u1_state(k) == s
        # words outside the block
        assert lay.shim_u1_index((1 << N) | 1) == -1
        if 0 < nup:
            assert lay.shim_u1_index((1 << (nup - 1)) - 1) == -1


@pytest.mark.parametrize("N,nup,L", [(24, 12, 12), (28, 14, 14), (32, 16, 16), (36, 18, 16), (40, 20, 16),
                                      (33, 5, 16), (20, 20, 10)])
def test_sampled_words_large_blocks(lay, orc, N, nup, L):
    dim, Lgot = _build(lay, N, nup)
    assert dim == math.comb(N, nup) and Lgot == L
    rng = np.random.default_rng(N + nup)
    for idx in list(rng.integers(0, dim, 300)) + [0, dim - 1]:
        s = orc.state_count(N, nup, int(idx))
        assert lay.shim_u1_state(int(idx)) == s
        assert lay.shim_u1_index(s) == int(idx) == orc.index_count(N, nup, s)

"""The library's host-side tridiagonal linear algebra (csrc/xd_tridiag.h:
Sturm bisection and inverse iteration for the Ritz values of T_m, Sec. 3.6.1;
cyclic Jacobi; exp(-z T_m) e_1 for the time evolution, Sec. 3.6.2) compiled
alone with g++ and checked against numpy / scipy."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_02901_gb300", "csrc")
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, f"libhosttridiag.{os.getpid()}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", so,
                           os.path.join(HERE, "host_tridiag_shim.cpp")])
    L = ctypes.CDLL(so)
    os.remove(so)
    L.shim_tridiag_eig.restype = ctypes.c_double
    L.shim_tridiag_eig.argtypes = [ctypes.c_int, D, D, ctypes.c_int]
    L.shim_tridiag_vec.argtypes = [ctypes.c_int, D, D, ctypes.c_double, D]
    L.shim_ritz.argtypes = [ctypes.c_int, D, D, ctypes.c_int, D, D]
    L.shim_jacobi.argtypes = [ctypes.c_int, D, D, D]
    L.shim_expm_e1.argtypes = [ctypes.c_int, D, D, ctypes.c_double, ctypes.c_double, D, D]
    return L


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(D)


def _T(d, e):
    return np.diag(d) + np.diag(e[: len(d) - 1], 1) + np.diag(e[: len(d) - 1], -1)


def _cases():
    rng = np.random.default_rng(0)
    out = []
    for n in (1, 2, 3, 10, 60, 150):
        out.append((rng.standard_normal(n), rng.uniform(0.1, 1.0, n)))
    n = 21  # Wilkinson W21+: pairs of nearly equal eigenvalues
    out.append((np.abs(np.arange(n) - 10.0), np.ones(n)))
    out.append((np.full(12, 2.0), np.r_[np.ones(5), 0.0, np.ones(6)]))  # split matrix, repeated spectrum
    out.append((np.linspace(-3, 3, 40), 1e-9 * np.ones(40)))  # almost diagonal
    return out


@pytest.mark.parametrize("case", range(9))
def test_sturm_bisection_and_inverse_iteration(lib, case):
    d, e = _cases()[case]
    d, e = _d(d), _d(e)
    n = len(d)
    T = _T(d, e)
    w = np.linalg.eigvalsh(T)
    scale = max(1.0, np.abs(w).max())
    for k in range(n):
        lam = lib.shim_tridiag_eig(n, _p(d), _p(e), k)
        assert abs(lam - w[k]) <= 1e-13 * scale, (k, lam, w[k])
        gap = min((abs(w[k] - w[j]) for j in (k - 1, k + 1) if 0 <= j < n), default=np.inf)
        if gap < 1e-9 * scale:
            continue  # (nearly) degenerate: the eigenvector is not unique
        z = _d(np.zeros(n))
        lib.shim_tridiag_vec(n, _p(d), _p(e), lam, _p(z))
        assert abs(np.linalg.norm(z) - 1) < 1e-12
        assert np.linalg.norm(T @ z - lam * z) < 1e-10 * scale
        first = np.flatnonzero(np.abs(z) > 1e-8)[0]
        assert z[first] > 0  # sign convention


def test_ritz_residuals(lib):
    rng = np.random.default_rng(5)
    n = 30
    a, b = _d(rng.standard_normal(n)), _d(rng.uniform(0.2, 1.0, n))
    ev, res = _d(np.zeros(3)), _d(np.zeros(3))
    lib.shim_ritz(n, _p(a), _p(b), 3, _p(ev), _p(res))
    w, V = np.linalg.eigh(_T(a, b))
    assert np.abs(ev - w[:3]).max() < 1e-12
    assert np.abs(res - np.abs(b[n - 1] * V[n - 1, :3])).max() < 1e-10


@pytest.mark.parametrize("n", [1, 2, 7, 40])
def test_jacobi(lib, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = _d(A + A.T)
    Q, w = _d(np.zeros((n, n))), _d(np.zeros(n))
    lib.shim_jacobi(n, _p(A), _p(Q), _p(w))
    assert np.abs(np.sort(w) - np.linalg.eigvalsh(A)).max() < 1e-12 * max(1, np.abs(w).max())
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-12
    assert np.abs(A @ Q - Q * w).max() < 1e-11 * max(1, np.abs(w).max())


@pytest.mark.parametrize("z", [0.7, 2.5j, 1.5 + 0.8j, 30.0])
def test_expm_e1(lib, z):
    from scipy.linalg import expm
    rng = np.random.default_rng(9)
    m = 25
    a, b = _d(rng.standard_normal(m) - 1.0), _d(rng.uniform(0.1, 1.0, m))
    cr, ci = _d(np.zeros(m)), _d(np.zeros(m))
    lib.shim_expm_e1(m, _p(a), _p(b), z.real if isinstance(z, complex) else z,
                     z.imag if isinstance(z, complex) else 0.0, _p(cr), _p(ci))
    want = expm(-z * _T(a, b))[:, 0]
    got = cr + 1j * ci
    assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())

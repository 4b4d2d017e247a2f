"""Python face of the CPU oracle (test infrastructure only).

The arithmetic lives in ``xd_oracle.c`` (plain C, FP64); this module builds
it with gcc, loads it with ctypes and adds the pieces that are library calls
in plain numpy: the Lanczos recurrence with full reorthogonalisation
(Sec. 3.6.1), dense matrices for full diagonalisation (Sec. 3.4) and the
Burnside count of symmetry-adapted block dimensions.

Nothing here imports the CUDA path, and the CUDA path never imports this.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile xd_oracle.c into _build/liboracle.so (OpenMP when available)."""
    src = os.path.join(_HERE, "xd_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(src)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    try:
        subprocess.check_call(base[:2] + ["-fopenmp"] + base[2:])
    except (subprocess.CalledProcessError, FileNotFoundError):
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32, _i64, _u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64


def _declare(L):
    sig = {
        "xo_threads": (_i32, [_i32]),
        "xo_binom": (_i64, [_i32, _i32]),
        "xo_popcount": (_i32, [_u64]),
        "xo_enumerate": (_i64, [_i32, _i32, _u64p]),
        "xo_index_search": (_i64, [_u64p, _i64, _u64]),
        "xo_index_count": (_i64, [_i32, _i32, _u64]),
        "xo_state_count": (_u64, [_i32, _i32, _i64]),
        "xo_splitmix64": (_u64, [_u64]),
        "xo_rng_normal": (ctypes.c_double, [_u64, _i64]),
        "xo_rng_fill": (None, [_u64, _i64, _i64, _f64p]),
        "xo_apply_u1": (None, [_i32, _u64p, _i64, _i32, _i32p, _f64p, _i32, _f64p, _f64p]),
        "xo_apply_rows_rng": (None, [_i32, _i32, _i32, _i32p, _f64p, _u64, _i64p, _i64, _f64p]),
        "xo_flip_index_rows": (None, [_i32, _i32, _i32, _i32p, _i64p, _i64, _i64p]),
        "xo_bond_forms": (None, [_i32, _u64p, _i64, _i32, _i32p, _f64p, _f64p, _f64p]),
        "xo_correlations": (None, [_i32, _u64p, _i64, _i32, _i32p, _i32, _f64p, _f64p]),
        "xo_act": (_u64, [_i32, _i32p, _u64]),
        "xo_group_check": (_i32, [_i32, _i32, _i32p, _f64p, _f64p]),
        "xo_rep": (_u64, [_i32, _i32, _i32p, _u64, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
        "xo_sym_basis": (_i64, [_i32, _i32, _i32, _i32p, _f64p, _f64p, _u64p, _i32p]),
        "xo_sym_apply": (None, [_i32, _i32, _i32p, _f64p, _f64p, _i32, _i32p, _f64p,
                                _u64p, _i32p, _i64, _f64p, _f64p]),
        "xo_keyed": (ctypes.c_double, [_u64, _u64, _i32]),
        "xo_sym_apply_rows_keyed": (None, [_i32, _i32, _i32p, _f64p, _f64p, _i32, _i32p, _f64p,
                                           _u64, _i32, _u64p, _i64, _f64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a, t):
    return a.ctypes.data_as(t)


def _bonds(bonds):
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    return b, b.shape[0]


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ------------------------------------------------------------------ basis
def threads(n: int = 0) -> int:
    """Threads of the oracle's OpenMP loops; n >= 1 sets them.  Returns the
    count in force."""
    return int(lib().xo_threads(n))


def binom(n: int, k: int) -> int:
    return int(lib().xo_binom(n, k))


def enumerate_states(N: int, nup: int) -> np.ndarray:
    """All N-bit words with nup ones, ascending (Sec. 3.1)."""
    n = lib().xo_enumerate(N, nup, None)
    if n < 0:
        raise ValueError("bad (N, nup)")
    out = np.empty(n, dtype=np.uint64)
    lib().xo_enumerate(N, nup, _p(out, _u64p))
    return out


def index_search(states: np.ndarray, s: int) -> int:
    return int(lib().xo_index_search(_p(states, _u64p), states.size, s))


def index_count(N: int, nup: int, s: int) -> int:
    return int(lib().xo_index_count(N, nup, s))


def state_count(N: int, nup: int, idx: int) -> int:
    return int(lib().xo_state_count(N, nup, idx))


# ------------------------------------------------------------------ random
def splitmix64(z: int) -> int:
    return int(lib().xo_splitmix64(z))


def rng_normal(seed: int, first: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    lib().xo_rng_fill(seed, first, n, _p(out, _f64p))
    return out


# ------------------------------------------------------------------ apply
def apply_u1(N: int, states: np.ndarray, bonds, J, x: np.ndarray) -> np.ndarray:
    """y = H x on a U(1) block; x is [dim] or [dim][nvec] (Eq. 1)."""
    b, nb = _bonds(bonds)
    J = _f64(J)
    x = _f64(x)
    nvec = 1 if x.ndim == 1 else x.shape[1]
    y = np.empty_like(x)
    lib().xo_apply_u1(N, _p(states, _u64p), states.size, nb, _p(b, _i32p), _p(J, _f64p),
                      nvec, _p(x, _f64p), _p(y, _f64p))
    return y


def apply_rows_rng(N: int, nup: int, bonds, J, seed: int, rows) -> np.ndarray:
    """Rows of H x for the unnormalised seeded normal x, with no stored list."""
    b, nb = _bonds(bonds)
    J = _f64(J)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    y = np.empty(rows.size, dtype=np.float64)
    lib().xo_apply_rows_rng(N, nup, nb, _p(b, _i32p), _p(J, _f64p), seed, _p(rows, _i64p),
                            rows.size, _p(y, _f64p))
    return y


def flip_index_rows(N: int, nup: int, bonds, rows) -> np.ndarray:
    b, nb = _bonds(bonds)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.empty((rows.size, nb), dtype=np.int64)
    lib().xo_flip_index_rows(N, nup, nb, _p(b, _i32p), _p(rows, _i64p), rows.size,
                             _p(out, _i64p))
    return out


def bond_forms(N: int, states: np.ndarray, bonds, g: np.ndarray, x: np.ndarray) -> np.ndarray:
    """out[b] = <g| S_i.S_j |x> for every bond (the J_b-derivative of <g|H|x>)."""
    b, nb = _bonds(bonds)
    g, x = _f64(g), _f64(x)
    out = np.empty(nb, dtype=np.float64)
    lib().xo_bond_forms(N, _p(states, _u64p), states.size, nb, _p(b, _i32p), _p(g, _f64p),
                        _p(x, _f64p), _p(out, _f64p))
    return out


def correlations(N: int, states: np.ndarray, pairs, kind: str, psi: np.ndarray) -> np.ndarray:
    """out[p] = <psi| O_{i_p j_p} |psi>, O = Sz_i Sz_j (kind "zz") or S_i.S_j
    (kind "ss"); i = j allowed."""
    b, n = _bonds(pairs)
    psi = _f64(psi)
    out = np.empty(n, dtype=np.float64)
    lib().xo_correlations(N, _p(states, _u64p), states.size, n, _p(b, _i32p),
                          {"zz": 0, "ss": 1}[kind], _p(psi, _f64p), _p(out, _f64p))
    return out


def dense_u1(N: int, states: np.ndarray, bonds, J) -> np.ndarray:
    """The block matrix, column by column from apply_u1 (small blocks only)."""
    dim = states.size
    return apply_u1(N, states, bonds, J, np.eye(dim))


# --------------------------------------------------------------- symmetry
def act(N: int, perm, s: int) -> int:
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    return int(lib().xo_act(N, _p(p, _i32p), s))


def group_check(N: int, perms, chi=None) -> int:
    p = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
    G = p.shape[0]
    if chi is None:
        return int(lib().xo_group_check(N, G, _p(p, _i32p), None, None))
    c = np.asarray(chi, dtype=np.complex128)
    cr, ci = _f64(c.real), _f64(c.imag)
    return int(lib().xo_group_check(N, G, _p(p, _i32p), _p(cr, _f64p), _p(ci, _f64p)))


def rep(N: int, perms, s: int):
    p = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
    u, cnt = ctypes.c_int(), ctypes.c_int()
    r = lib().xo_rep(N, p.shape[0], _p(p, _i32p), s, ctypes.byref(u), ctypes.byref(cnt))
    return int(r), u.value, cnt.value


def keyed(seed: int, words, cplx: bool = False) -> np.ndarray:
    """x_w = xo_keyed(seed, w, 0) (+ i xo_keyed(seed, w, 1)) for each word."""
    f = lib().xo_keyed
    re = np.array([f(seed, int(w), 0) for w in words])
    if not cplx:
        return re
    return re + 1j * np.array([f(seed, int(w), 1) for w in words])


def sym_apply_rows_keyed(N: int, perms, chi, bonds, J, seed: int, cplx: bool, rows) -> np.ndarray:
    """Rows (given by their representatives) of H x on a symmetry-adapted
    block, x keyed on the representatives (xo_sym_apply_rows_keyed)."""
    p = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
    c = np.asarray(chi, dtype=np.complex128)
    cr, ci = _f64(c.real), _f64(c.imag)
    b, nb = _bonds(bonds)
    Jv = _f64(J)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.uint64))
    y = np.empty(r.size, dtype=np.complex128)
    lib().xo_sym_apply_rows_keyed(N, p.shape[0], _p(p, _i32p), _p(cr, _f64p), _p(ci, _f64p), nb, _p(b, _i32p),
                                  _p(Jv, _f64p), seed, 1 if cplx else 0, _p(r, _u64p), r.size,
                                  _p(y.view(np.float64), _f64p))
    return y


class SymBlock:
    """Symmetry-adapted U(1) block (Sec. 3.10): representatives and |Stab|."""

    def __init__(self, N, nup, perms, chi):
        self.N, self.nup = N, nup
        self.perms = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
        c = np.asarray(chi, dtype=np.complex128)
        self.chi = c
        self._cr, self._ci = _f64(c.real), _f64(c.imag)
        G = self.perms.shape[0]
        rc = group_check(N, self.perms, c)
        if rc:
            raise ValueError(f"invalid group/representation (code {rc})")
        n = lib().xo_sym_basis(N, nup, G, _p(self.perms, _i32p), _p(self._cr, _f64p),
                               _p(self._ci, _f64p), None, None)
        self.reps = np.empty(n, dtype=np.uint64)
        self.stab = np.empty(n, dtype=np.int32)
        lib().xo_sym_basis(N, nup, G, _p(self.perms, _i32p), _p(self._cr, _f64p),
                           _p(self._ci, _f64p), _p(self.reps, _u64p), _p(self.stab, _i32p))

    @property
    def dim(self):
        return self.reps.size

    def apply(self, bonds, J, x):
        b, nb = _bonds(bonds)
        J = _f64(J)
        xc = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        y = np.empty_like(xc)
        xv, yv = xc.view(np.float64), y.view(np.float64)
        lib().xo_sym_apply(self.N, self.perms.shape[0], _p(self.perms, _i32p),
                           _p(self._cr, _f64p), _p(self._ci, _f64p), nb, _p(b, _i32p),
                           _p(J, _f64p), _p(self.reps, _u64p), _p(self.stab, _i32p),
                           self.dim, _p(xv, _f64p), _p(yv, _f64p))
        return y

    def dense(self, bonds, J):
        """The block's matrix, column k = (block product of unit vector k)."""
        return np.stack([self.apply(bonds, J, e) for e in np.eye(self.dim, dtype=np.complex128)], axis=1)

    def lift(self, states: np.ndarray) -> np.ndarray:
        """Columns |r_chi> = N_r^-1 sum_g conj(chi(g)) g|r> in the U(1) basis."""
        G = self.perms.shape[0]
        B = np.zeros((states.size, self.dim), dtype=np.complex128)
        for k, r in enumerate(self.reps):
            col = np.zeros(states.size, dtype=np.complex128)
            for g in range(G):
                t = act(self.N, self.perms[g], int(r))
                col[index_search(states, t)] += np.conj(self.chi[g])
            B[:, k] = col / math.sqrt(G * int(self.stab[k]))
        return B


def project(N: int, perms, chi, s: int, states: np.ndarray) -> np.ndarray:
    """N^-1 sum_g conj(chi(g)) g|s> for any product state s (Sec. 3.10)."""
    perms = np.asarray(perms, dtype=np.int32)
    v = np.zeros(states.size, dtype=np.complex128)
    for g in range(perms.shape[0]):
        v[index_search(states, act(N, perms[g], s))] += np.conj(chi[g])
    return v / np.linalg.norm(v)


def burnside_dim(N: int, nup: int, perms, chi) -> int:
    """dim of the chi block = (1/|G|) sum_g conj(chi(g)) Fix_nup(g), where
    Fix_nup(g) counts words with nup ones fixed by g: constant on each cycle
    of g, so the cycle lengths must sum to nup (subset-sum count)."""
    perms = np.asarray(perms, dtype=np.int64)
    total = 0j
    for g in range(perms.shape[0]):
        seen = [False] * N
        lens = []
        for i in range(N):
            if not seen[i]:
                L, j = 0, i
                while not seen[j]:
                    seen[j] = True
                    j = int(perms[g, j])
                    L += 1
                lens.append(L)
        ways = [0] * (nup + 1)
        ways[0] = 1
        for L in lens:
            for t in range(nup, L - 1, -1):
                ways[t] += ways[t - L]
        total += np.conj(chi[g]) * ways[nup]
    val = total / perms.shape[0]
    assert abs(val.imag) < 1e-6 and abs(val.real - round(val.real)) < 1e-6
    return int(round(val.real))


# ---------------------------------------------------------------- Lanczos
def lanczos(matvec, dim: int, v0: np.ndarray, steps: int, full_reorth: bool = True,
            tol: float = 1e-13):
    """Lanczos tridiagonalisation (Sec. 3.6.1) in FP64 from the start v0.

    Returns (alpha, beta) with T = tridiag(beta[:-1], alpha, beta[:-1]).
    Complex vectors (the blocks of complex characters) take the Hermitian
    inner product <v|w>, which is real for a Hermitian H.  With full_reorth
    the new vector is orthogonalised against all earlier ones twice
    (classical Gram-Schmidt, repeated)."""
    v0 = np.asarray(v0)
    v = v0.astype(np.complex128 if np.iscomplexobj(v0) else np.float64) / np.linalg.norm(v0)
    V = [v]
    alpha, beta = [], []
    b_prev, v_prev = 0.0, np.zeros_like(v)
    for k in range(steps):
        w = matvec(v) - b_prev * v_prev
        a = float(np.vdot(v, w).real)
        w = w - a * v
        if full_reorth:
            for _ in range(2):
                Vm = np.array(V)
                w = w - Vm.T @ (Vm.conj() @ w)
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        if b < tol * max(abs(t) for t in alpha) or k == steps - 1:
            break
        v_prev, v = v, w / b
        b_prev = b
        if full_reorth:
            V.append(v)
    return np.array(alpha), np.array(beta)


def tridiag_eigvals(alpha, beta) -> np.ndarray:
    """Eigenvalues of the symmetric tridiagonal T (numpy eigh)."""
    n = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: n - 1], 1) + np.diag(beta[: n - 1], -1)
    return np.linalg.eigvalsh(T)


def lanczos_ground_state(matvec, dim, v0, steps, full_reorth=True):
    """Ground energy and vector: Lanczos run, then the Ritz vector sum c_k v_k
    rebuilt from a second run with the same start (eig0, Sec. 3.6.1)."""
    alpha, beta = lanczos(matvec, dim, v0, steps, full_reorth)
    n = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: n - 1], 1) + np.diag(beta[: n - 1], -1)
    w, Q = np.linalg.eigh(T)
    c = Q[:, 0]
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    V = [v]
    psi = c[0] * v
    b_prev, v_prev = 0.0, np.zeros_like(v)
    for k in range(n - 1):
        w_ = matvec(v) - b_prev * v_prev - alpha[k] * v
        if full_reorth:
            for _ in range(2):
                Vm = np.array(V)
                w_ = w_ - Vm.T @ (Vm @ w_)
        v_prev, v = v, w_ / beta[k]
        b_prev = beta[k]
        V.append(v)
        psi = psi + c[k + 1] * v
    psi = psi / np.linalg.norm(psi)
    return float(w[0]), psi


# ----------------------------------------------------------- time evolution
def evolve_dense(H: np.ndarray, psi0: np.ndarray, z: complex) -> np.ndarray:
    """exp(-z H) psi0 for a dense Hermitian block H (Sec. 3.6.2: z = i t gives
    the real-time evolution e^{-iHt}, z = tau the imaginary-time e^{-tau H}),
    written out through the eigendecomposition H = V diag(w) V^dagger."""
    w, V = np.linalg.eigh(H)
    return V @ (np.exp(-z * w) * (V.conj().T @ np.asarray(psi0, dtype=np.complex128)))


# ------------------------------------------------------------ thermodynamics
def ftlm_tridiagonals(matvec, starts, steps: int):
    """Finite-temperature Lanczos (the thermal pure quantum state / FTLM
    ensemble of the paper's thermodynamics examples): one plain Lanczos run
    (no reorthogonalisation) per start vector r, returning the lists of
    (alpha, beta) and the norms |r|."""
    out = []
    for r in starts:
        a, b = lanczos(matvec, r.size, r, steps, full_reorth=False, tol=0.0)
        out.append((a, b, float(np.linalg.norm(r))))
    return out


def ftlm_thermo(tri, dim: int, temps, exact_trace: bool = False):
    """Z, E and C at the temperatures T from the tridiagonals T_r:
    T_r = Q diag(eps) Q^T, weights |Q_0j|^2, and with R starts
        Z = (dim / R) sum_r sum_j |Q_0j|^2 e^{-eps_j / T}
        E = (dim / R) sum ... eps_j e^{-eps_j/T} / Z,  C = (<E^2> - E^2) / T^2.
    Random starts are normalised to unit length; with exact_trace the starts
    are taken as given (an orthonormal basis gives the trace exactly, so the
    prefactor dim / R is then 1)."""
    R = len(tri)
    pref = 1.0 if exact_trace else dim / R
    res = []
    for T in temps:
        z = e1 = e2 = 0.0
        shift = min(np.linalg.eigvalsh(_tri(a, b)).min() for a, b, _ in tri)
        for a, b, nr in tri:
            w, Q = np.linalg.eigh(_tri(a, b))
            wt = Q[0, :] ** 2 * np.exp(-(w - shift) / T)
            z += wt.sum()
            e1 += (w * wt).sum()
            e2 += (w * w * wt).sum()
        E = e1 / z
        res.append((pref * z * np.exp(-shift / T), E, (e2 / z - E * E) / T ** 2))
    return res


def _tri(a, b):
    n = len(a)
    return np.diag(a) + np.diag(b[: n - 1], 1) + np.diag(b[: n - 1], -1)

"""PyTorch face of the CUDA library: blocks, Hamiltonians, Lanczos, autograd.

Tensors are device memory and streams only; every step of H x, the
bilinear forms, the Lanczos vector updates and the batched product runs in
libxdgpu.so.  Calls go to the current torch CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import XD_C128, XD_EINVAL, XD_F32, XD_F64, XDError, check

_DT = {torch.float64: XD_F64, torch.float32: XD_F32, torch.complex128: XD_C128}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return _DT[t.dtype]


def _check_vec(t: torch.Tensor, dim: int, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.shape[0] != dim:
        raise ValueError(f"{name} has {t.shape[0]} rows, the block has {dim}")


class Basis:
    """Spinhalf(N, nup[, irrep]) block on an interaction graph (Sec. 3.1, 3.10)."""

    def __init__(self, N: int, nup: int, bonds, symmetry=None):
        L = _lib.lib()
        b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        self.N, self.nup, self.bonds = int(N), int(nup), b
        self._h = ctypes.c_void_p()
        sym_p = None
        if symmetry is not None:
            perms, chi = symmetry
            self._perms = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
            c = np.asarray(chi, dtype=np.complex128)
            self._cr = np.ascontiguousarray(c.real)
            self._ci = np.ascontiguousarray(c.imag)
            sym = _lib.xd_symmetry(self._perms.shape[0],
                                   self._perms.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   self._cr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   self._ci.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
            sym_p = ctypes.byref(sym)
        check(L.xd_basis_create(self.N, self.nup,
                                b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), b.shape[0],
                                sym_p, ctypes.byref(self._h)))
        d = ctypes.c_int64()
        check(L.xd_basis_dim(self._h, ctypes.byref(d)))
        self.dim = int(d.value)
        c = ctypes.c_int()
        check(L.xd_basis_is_complex(self._h, ctypes.byref(c)))
        self.is_complex = bool(c.value)
        self.symmetric = symmetry is not None

    @property
    def nb(self):
        return self.bonds.shape[0]

    def state(self, idx: int) -> int:
        s = ctypes.c_uint64()
        check(_lib.lib().xd_basis_state(self._h, int(idx), ctypes.byref(s)))
        return int(s.value)

    def index(self, s: int) -> int:
        i = ctypes.c_int64()
        check(_lib.lib().xd_basis_index(self._h, int(s), ctypes.byref(i)))
        return int(i.value)

    def states(self, first: int = 0, count: int | None = None) -> torch.Tensor:
        """State words of rows [first, first + count) (representatives on a
        symmetric block) as a CUDA int64 tensor."""
        count = self.dim - first if count is None else int(count)
        out = torch.empty(max(count, 0), dtype=torch.int64, device="cuda")
        check(_lib.lib().xd_basis_states(self._h, int(first), count, _ptr(out), _stream()))
        return out

    def correlations(self, psi: torch.Tensor, pairs, kind: str = "ss") -> np.ndarray:
        """<psi| O_ij |psi> for every site pair, O = S_i.S_j (kind "ss") or
        Sz_i Sz_j (kind "zz") (Sec. 3.7 inner), on U(1) and symmetry-adapted
        blocks (the lifted state's values; xd_correlations)."""
        _check_vec(psi, self.dim, "psi")
        if kind not in ("zz", "ss"):
            raise XDError(XD_EINVAL, f"correlations: kind must be 'zz' or 'ss', not {kind!r}")
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        out = np.zeros(p.shape[0])
        torch.cuda.current_stream().synchronize()
        check(_lib.lib().xd_correlations(self._h, _ptr(psi), _dtype_code(psi),
                                         p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), p.shape[0],
                                         {"zz": 0, "ss": 1}[kind], out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.xd_basis_destroy(h)
            self._h = None


class Hamiltonian:
    """H = sum_b J_b S_i.S_j on a Basis (Eq. 1)."""

    def __init__(self, basis: Basis, J):
        self.basis = basis
        self._h = ctypes.c_void_p()
        self.J = np.ascontiguousarray(np.asarray(J, dtype=np.float64))
        check(_lib.lib().xd_ham_create(basis._h, self.J.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(self._h)))

    @property
    def dim(self):
        return self.basis.dim

    def set_couplings(self, J):
        J = np.ascontiguousarray(np.asarray(J, dtype=np.float64))
        check(_lib.lib().xd_ham_set_couplings(self._h, J.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        self.J = J

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = H x; x is [dim] or [dim, nvec] (float64, float32 or complex128)."""
        _check_vec(x, self.dim, "x")
        nvec = 1 if x.dim() == 1 else x.shape[1]
        y = torch.empty_like(x) if out is None else out
        _check_vec(y, self.dim, "out")
        check(_lib.lib().xd_apply(self._h, _ptr(x), _ptr(y), _dtype_code(x), nvec, _stream()))
        return y

    def bilinear(self, g: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        """dJ[b] = Re <g| S_i.S_j |x> for every bond (device float64 [nb]);
        for [dim, nvec] g and x, the sum over the columns."""
        _check_vec(g, self.dim, "g")
        _check_vec(x, self.dim, "x")
        if g.dtype != x.dtype or g.shape != x.shape:
            raise TypeError("g and x must have the same dtype and shape")
        nvec = 1 if x.dim() == 1 else x.shape[1]
        out = torch.empty(self.basis.nb, dtype=torch.float64, device=x.device)
        check(_lib.lib().xd_apply_bilinear_nvec(self._h, _ptr(g), _ptr(x), _dtype_code(x), nvec, _ptr(out),
                                                _stream()))
        return out

    def _lanczos(self, max_iter, seed, storage, nev, psi=None):
        dt = _DT[storage]
        a = np.zeros(max_iter)
        b = np.zeros(max_iter)
        n = ctypes.c_int()
        ev = np.zeros(nev)
        rs = np.zeros(nev)
        P = lambda arr: arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        torch.cuda.current_stream().synchronize()
        if psi is None:
            check(_lib.lib().xd_lanczos_eigenvalues(self._h, max_iter, seed, dt, nev, P(a), P(b),
                                                    ctypes.byref(n), P(ev), P(rs)))
        else:
            check(_lib.lib().xd_lanczos_ground_state(self._h, max_iter, seed, dt, nev, P(a), P(b),
                                                     ctypes.byref(n), P(ev), P(rs), _ptr(psi)))
        k = n.value
        return dict(alpha=a[:k], beta=b[:k], n_iter=k, evals=ev, resid=rs)

    def lanczos(self, max_iter=200, seed=1, storage=torch.float64, nev=1):
        """Lanczos eigenvalues (eigvals_lanczos, Sec. 3.6.1)."""
        return self._lanczos(max_iter, seed, storage, nev)

    def ground_state(self, max_iter=200, seed=1, storage=torch.float64, nev=1):
        """(E0, psi0, info) by two Lanczos passes (eig0, Sec. 3.6.1)."""
        if self.basis.is_complex:
            storage = torch.complex128
        psi = torch.empty(self.dim, dtype=storage, device="cuda")
        info = self._lanczos(max_iter, seed, storage, nev, psi)
        return float(info["evals"][0]), psi, info

    def evolve(self, psi0: torch.Tensor, t: float = 0.0, tau: float = 0.0, max_iter: int = 200,
               tol: float = 1e-12):
        """exp(-(tau + i t) H) psi0 (Sec. 3.6.2 time_evolve: real time t,
        imaginary time tau) by the two-pass Lanczos method.  psi0: complex128
        CUDA tensor [dim].  Returns (psi, {"n_iter", "err"})."""
        _check_vec(psi0, self.dim, "psi0")
        if psi0.dtype != torch.complex128:
            raise TypeError("psi0 must be complex128")
        out = torch.empty_like(psi0)
        n = ctypes.c_int()
        err = ctypes.c_double()
        torch.cuda.current_stream().synchronize()
        check(_lib.lib().xd_evolve(self._h, _ptr(psi0), float(tau), float(t), int(max_iter), float(tol),
                                   _ptr(out), ctypes.byref(n), ctypes.byref(err)))
        return out, {"n_iter": n.value, "err": err.value}

    def ftlm(self, R: int = 16, M: int = 80, seed: int = 1):
        """Finite-temperature Lanczos tridiagonals of R random starts (seed + r),
        M steps each; returns (alpha [R, M], beta [R, M], n_iter [R]) (xd_ftlm:
        U(1) blocks eight starts at a time on the eight-vector product,
        symmetry-adapted blocks one Lanczos pass per start)."""
        if R < 1 or M < 1:
            raise XDError(XD_EINVAL, "ftlm: need R >= 1 and M >= 1")
        a = np.zeros((R, M))
        b = np.zeros((R, M))
        n = np.zeros(R, dtype=np.int32)
        torch.cuda.current_stream().synchronize()
        dp = ctypes.POINTER(ctypes.c_double)
        check(_lib.lib().xd_ftlm(self._h, int(R), int(M), ctypes.c_uint64(seed), a.ctypes.data_as(dp),
                                 b.ctypes.data_as(dp), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return a, b, n

    def energy_grad(self, psi0: torch.Tensor) -> np.ndarray:
        """dE0/dJ_b = <psi0|S_i.S_j|psi0> (Hellmann-Feynman, Sec. 3.7 inner)."""
        _check_vec(psi0, self.dim, "psi0")
        out = np.zeros(self.basis.nb)
        torch.cuda.current_stream().synchronize()
        check(_lib.lib().xd_energy_grad(self._h, _ptr(psi0), _dtype_code(psi0),
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.xd_ham_destroy(h)
            self._h = None


def ftlm_thermo(alpha: np.ndarray, beta: np.ndarray, n_iter: np.ndarray, dim: int, temps):
    """(Z, E, C) at the temperatures from the tridiagonals of Hamiltonian.ftlm."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    n_iter = np.ascontiguousarray(n_iter, dtype=np.int32)
    T = np.ascontiguousarray(np.asarray(temps, dtype=np.float64).reshape(-1))
    Z, E, C = np.zeros(T.size), np.zeros(T.size), np.zeros(T.size)
    dp = ctypes.POINTER(ctypes.c_double)
    check(_lib.lib().xd_ftlm_thermo(alpha.shape[0], alpha.shape[1], alpha.ctypes.data_as(dp), beta.ctypes.data_as(dp),
                                    n_iter.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(dim), T.size,
                                    T.ctypes.data_as(dp), Z.ctypes.data_as(dp), E.ctypes.data_as(dp),
                                    C.ctypes.data_as(dp)))
    return Z, E, C


def random_vector(dim: int, seed: int, dtype=torch.float64, out=None) -> torch.Tensor:
    """Seeded N(0,1) vector (unnormalised) from the library's counter RNG."""
    v = torch.empty(dim, dtype=dtype, device="cuda") if out is None else out
    check(_lib.lib().xd_random_vector(dim, seed, _ptr(v), _DT[v.dtype], _stream()))
    return v


def batch_apply(hams, xs, ys) -> None:
    """ys[k] = H_k xs[k] for every k in one persistent, graph-replayed launch."""
    n = len(hams)
    if not (n == len(xs) == len(ys)) or n == 0:
        raise ValueError("hams, xs, ys must be non-empty and of equal length")
    dt = _dtype_code(xs[0])
    nvec = 1 if xs[0].dim() == 1 else xs[0].shape[1]
    for h, x, y in zip(hams, xs, ys):
        _check_vec(x, h.dim, "x")
        _check_vec(y, h.dim, "y")
        if x.dtype != xs[0].dtype or y.dtype != xs[0].dtype:
            raise TypeError("all vectors must share one dtype")
    H = (ctypes.c_void_p * n)(*[h._h.value for h in hams])
    X = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    Y = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    check(_lib.lib().xd_batch_apply(n, H, X, Y, dt, nvec, _stream()))


class HeisenbergApply(torch.autograd.Function):
    """y = H(J) x with backward dL/dx = H g (H real symmetric) and
    dL/dJ_b = sum_r g_r (S_i.S_j x)_r (the bilinear kernel)."""

    @staticmethod
    def forward(ctx, J, x, ham):
        Jn = J.detach().to("cpu", torch.float64).numpy()
        if not np.array_equal(Jn, ham.J):
            ham.set_couplings(Jn)
        ctx.ham = ham
        ctx.jdev = J.device
        ctx.save_for_backward(x)
        return ham.apply(x.contiguous())

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        ham = ctx.ham
        g = g.contiguous()
        gx = ham.apply(g) if ctx.needs_input_grad[1] else None
        gJ = ham.bilinear(g, x.contiguous()).to(ctx.jdev) if ctx.needs_input_grad[0] else None
        return gJ, gx, None


def heisenberg_apply(ham: Hamiltonian, J: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    return HeisenbergApply.apply(J, x, ham)


class GroundEnergy(torch.autograd.Function):
    """E0(J) by Lanczos; backward dE0/dJ_b = <psi0|S_i.S_j|psi0>."""

    @staticmethod
    def forward(ctx, J, ham, max_iter, seed, storage):
        Jn = J.detach().to("cpu", torch.float64).numpy()
        if not np.array_equal(Jn, ham.J):
            ham.set_couplings(Jn)
        e0, psi, _ = ham.ground_state(max_iter, seed, storage)
        ctx.grad = torch.from_numpy(ham.energy_grad(psi)).to(J.device)
        return torch.tensor(e0, dtype=torch.float64, device=J.device)

    @staticmethod
    def backward(ctx, g):
        return g * ctx.grad, None, None, None, None


def ground_energy(ham: Hamiltonian, J: torch.Tensor, max_iter=200, seed=1, storage=torch.float64):
    return GroundEnergy.apply(J, ham, max_iter, seed, storage)


__all__ = ["Basis", "Hamiltonian", "random_vector", "batch_apply", "heisenberg_apply",
           "ground_energy", "HeisenbergApply", "GroundEnergy", "XDError", "ftlm_thermo"]

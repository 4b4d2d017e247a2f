"""Seeded synthetic inputs: lattices, couplings and symmetry groups.

This module holds no arithmetic of the method.  It only produces the inputs
that both the CUDA path and the CPU oracle receive: bond lists, coupling
values drawn from a seed, site permutations of translation groups and the
characters of their one-dimensional irreps.

Site labelling: a rectangular Lx x Ly lattice numbers site (x, y) as
i = x + Lx*y, periodic in both directions.  Bit i of a state word is site i.
"""
from __future__ import annotations

import cmath
import math

import numpy as np


def _dedupe(pairs):
    seen, out = set(), []
    for i, j in pairs:
        if i == j:
            continue
        key = (min(i, j), max(i, j))
        if key in seen:
            continue
        seen.add(key)
        out.append((i, j))
    return out


def chain(N: int) -> np.ndarray:
    """Periodic chain bonds (i, i+1 mod N) (Sec. 3.2 and its TOML listing in
    Sec. 3.8); for N = 2 the two periodic bonds are the same pair, kept once."""
    return np.array(_dedupe([(i, (i + 1) % N) for i in range(N)]), dtype=np.int32)


def chain_j1j2(N: int, J1: float = 1.0, J2: float = 0.5):
    """Periodic chain with nearest (J1) and next-nearest (J2) neighbour bonds,
    J1 bonds (i, i+1) first, then (i, i+2).  J2 = J1/2 is the Majumdar-Ghosh
    point.  Returns (bonds [2N, 2] int32, J [2N])."""
    if N < 5:
        raise ValueError("the J1-J2 chain needs N >= 5 for distinct bonds")
    b = [(i, (i + 1) % N) for i in range(N)] + [(i, (i + 2) % N) for i in range(N)]
    return np.array(b, dtype=np.int32), np.array([J1] * N + [J2] * N, dtype=np.float64)


def ladder(L: int, rung_copies: int = 2) -> np.ndarray:
    """Two-leg periodic ladder on the L x 2 lattice (leg y=0 is sites 0..L-1,
    leg y=1 is sites L..2L-1).  Bond order: leg 0 (i, i+1), leg 1, then the
    rungs (i, i+L) once per copy.  rung_copies=2 is what a periodic L x 2
    square-lattice generator produces (each rung listed twice, 4L bonds, 56
    for L=14); rung_copies=1 gives the 3L-bond ladder."""
    b = [(i, (i + 1) % L) for i in range(L)]
    b += [(L + i, L + (i + 1) % L) for i in range(L)]
    for _ in range(rung_copies):
        b += [(i, i + L) for i in range(L)]
    return np.array(b, dtype=np.int32)


def square_j1j2(Lx: int, Ly: int, J1: float = 1.0, J2: float = 0.5):
    """Periodic Lx x Ly square lattice: J1 on (x+1, y) and (x, y+1), J2 on
    (x+1, y+1) and (x-1, y+1).  Each unordered pair kept once.  Returns
    (bonds [nb, 2] int32, J [nb] float64), J1 bonds first."""
    s = lambda x, y: (x % Lx) + Lx * (y % Ly)  # noqa: E731
    nn = _dedupe([(s(x, y), s(x + 1, y)) for y in range(Ly) for x in range(Lx)]
                 + [(s(x, y), s(x, y + 1)) for y in range(Ly) for x in range(Lx)])
    nnn = _dedupe([(s(x, y), s(x + 1, y + 1)) for y in range(Ly) for x in range(Lx)]
                  + [(s(x, y), s(x - 1, y + 1)) for y in range(Ly) for x in range(Lx)])
    nnn = [p for p in nnn if (min(p), max(p)) not in {(min(q), max(q)) for q in nn}]
    bonds = np.array(nn + nnn, dtype=np.int32)
    J = np.array([J1] * len(nn) + [J2] * len(nnn), dtype=np.float64)
    return bonds, J


def uniform_couplings(nb: int, seed: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """J_b ~ U[lo, hi) from numpy's PCG64 stream seeded with `seed`."""
    return np.random.default_rng(seed).uniform(lo, hi, size=nb).astype(np.float64)


def random_bonds(N: int, nb: int, seed: int) -> np.ndarray:
    """nb distinct random site pairs (for parity tests on irregular graphs)."""
    rng = np.random.default_rng(seed)
    pairs = set()
    out = []
    while len(out) < nb:
        i, j = (int(v) for v in rng.integers(0, N, size=2))
        if i == j or (min(i, j), max(i, j)) in pairs:
            continue
        pairs.add((min(i, j), max(i, j)))
        out.append((i, j))
    return np.array(out, dtype=np.int32)


# ------------------------------------------------------------- symmetry
def chain_translations(N: int) -> np.ndarray:
    """perms[n][i] = (i + n) mod N, the powers T^n of the chain translation."""
    return np.array([[(i + n) % N for i in range(N)] for n in range(N)], dtype=np.int32)


def chain_dihedral(N: int) -> np.ndarray:
    """The dihedral group D_N of the periodic chain: perms[n][i] = (i + n) mod N
    (translations T^n), then perms[N + n][i] = (n - i) mod N (reflections)."""
    rot = [[(i + n) % N for i in range(N)] for n in range(N)]
    ref = [[(n - i) % N for i in range(N)] for n in range(N)]
    return np.array(rot + ref, dtype=np.int32)


def chain_dihedral_characters(N: int, m: int, parity: int) -> np.ndarray:
    """One-dimensional characters of D_N (Sec. 3.9.2): momentum k = 2 pi m / N
    with k in {0, pi}, chi(T^n) = exp(i k n), chi(reflection n) = parity exp(i k n)."""
    if (2 * m) % N != 0 or parity not in (1, -1):
        raise ValueError("D_N has one-dimensional irreps only at k = 0, pi and parity +-1")
    k = 2 * math.pi * m / N
    rot = [cmath.exp(1j * k * n) for n in range(N)]
    return np.array(rot + [parity * z for z in rot], dtype=np.complex128)


def torus_space_group(L: int) -> np.ndarray:
    """Space group of the periodic L x L square lattice: the 8 point operations
    of the square (rotations by 90 degrees and mirrors) followed by the L^2
    translations, perms[g][i] = site of op(x, y) + (a, b), 8 L^2 elements."""
    ops = [lambda x, y: (x, y), lambda x, y: (-y, x), lambda x, y: (-x, -y), lambda x, y: (y, -x),
           lambda x, y: (-x, y), lambda x, y: (x, -y), lambda x, y: (y, x), lambda x, y: (-y, -x)]
    out = []
    for op in ops:
        for b in range(L):
            for a in range(L):
                row = []
                for i in range(L * L):
                    x, y = op(i % L, i // L)
                    row.append((x + a) % L + L * ((y + b) % L))
                out.append(row)
    return np.array(out, dtype=np.int32)


# Point groups in lattice coordinates: generated by a rotation R of order n
# and a mirror M, elements R^k M^e (e = 0, 1; k = 0 .. n-1), as integer 2x2
# matrices acting on (x, y).
POINT_GROUPS = {
    "square": ((0, -1, 1, 0), 4, (-1, 0, 0, 1)),       # C4v: 90-degree rotation, x -> -x
    "rectangular": ((-1, 0, 0, -1), 2, (-1, 0, 0, 1)),  # C2v: 180-degree rotation, x -> -x
    # C6v of the triangular lattice with primitive vectors a1 = (1, 0),
    # a2 = (1/2, sqrt(3)/2): the 60-degree rotation maps a1 -> a2 -> a2 - a1,
    # the mirror swaps a1 and a2
    "triangular": ((0, -1, 1, 1), 6, (0, 1, 1, 0)),
}


def _mat(m, x, y):
    return m[0] * x + m[1] * y, m[2] * x + m[3] * y


def space_group(Lx: int, Ly: int, lattice: str) -> np.ndarray:
    """Translations times a point group on the periodic Lx x Ly lattice (site
    x + Lx*y).  Element (e, k, b, a) = T_{a,b} R^k M^e, listed e-major, then k,
    b, a: perms[g][i] = site of R^k M^e (x, y) + (a, b); n 2 Lx Ly elements.
    The point operations must map the torus onto itself (Lx = Ly for the
    square and triangular groups)."""
    R, n, M = POINT_GROUPS[lattice]
    if lattice != "rectangular" and Lx != Ly:
        raise ValueError(f"the {lattice} point group needs Lx == Ly")
    out = []
    for e in range(2):
        for k in range(n):
            for b in range(Ly):
                for a in range(Lx):
                    row = []
                    for i in range(Lx * Ly):
                        x, y = i % Lx, i // Lx
                        if e:
                            x, y = _mat(M, x, y)
                        for _ in range(k):
                            x, y = _mat(R, x, y)
                        row.append((x + a) % Lx + Lx * ((y + b) % Ly))
                    out.append(row)
    return np.array(out, dtype=np.int32)


def space_group_characters(Lx: int, Ly: int, lattice: str, r: int = 1, m: int = 1,
                           mx: int = 0, my: int = 0) -> np.ndarray:
    """One-dimensional characters of space_group(Lx, Ly, lattice):
    chi(T_{a,b} R^k M^e) = r^k m^e exp(i (kx a + ky b)) with r, m = +-1 and
    momentum (kx, ky) = (2 pi mx / Lx, 2 pi my / Ly), which must be left
    invariant by the point group (Gamma; M = (pi, pi) on the square lattice).
    r = -1 needs an even rotation order; r = m = 1 is the fully symmetric A1."""
    _, n, _ = POINT_GROUPS[lattice]
    kx, ky = 2 * math.pi * mx / Lx, 2 * math.pi * my / Ly
    out = []
    for e in range(2):
        for k in range(n):
            for b in range(Ly):
                for a in range(Lx):
                    z = (r ** k) * (m ** e) * cmath.exp(1j * (kx * a + ky * b))
                    out.append(complex(round(z.real, 15), round(z.imag, 15)))
    return np.array(out, dtype=np.complex128)


def triangular(L: int, J1: float = 1.0) -> tuple:
    """Periodic L x L triangular lattice in the coordinates of a1 = (1, 0),
    a2 = (1/2, sqrt(3)/2): bonds to (x+1, y), (x, y+1), (x-1, y+1), each
    unordered pair kept once.  Returns (bonds [nb, 2] int32, J [nb])."""
    s = lambda x, y: (x % L) + L * (y % L)  # noqa: E731
    b = _dedupe([(s(x, y), s(x + 1, y)) for y in range(L) for x in range(L)]
                + [(s(x, y), s(x, y + 1)) for y in range(L) for x in range(L)]
                + [(s(x, y), s(x - 1, y + 1)) for y in range(L) for x in range(L)])
    return np.array(b, dtype=np.int32), np.full(len(b), J1)


def shastry_sutherland(Lx: int, Ly: int, J: float = 1.0, Jp: float = 0.5):
    """Shastry-Sutherland lattice on the periodic Lx x Ly square lattice (Lx,
    Ly even), the model of the paper's thermal pure quantum state example
    (Sec. 4): nearest-neighbour bonds J' and orthogonal dimers J on half of
    the plaquette diagonals, (x, y)-(x+1, y+1) for x, y even and
    (x+1, y)-(x, y+1) for x, y odd, so that every site is in one dimer.
    Returns (bonds [nb, 2] int32, J [nb], dimers [N/2, 2] int32); the dimer
    bonds come first."""
    if Lx % 2 or Ly % 2 or Lx < 4 or Ly < 4:
        raise ValueError("the Shastry-Sutherland pattern needs even Lx, Ly >= 4")
    s = lambda x, y: (x % Lx) + Lx * (y % Ly)  # noqa: E731
    dim = []
    for y in range(Ly):
        for x in range(Lx):
            if x % 2 == 0 and y % 2 == 0:
                dim.append((s(x, y), s(x + 1, y + 1)))
            elif x % 2 == 1 and y % 2 == 1:
                dim.append((s(x + 1, y), s(x, y + 1)))
    nn = _dedupe([(s(x, y), s(x + 1, y)) for y in range(Ly) for x in range(Lx)]
                 + [(s(x, y), s(x, y + 1)) for y in range(Ly) for x in range(Lx)])
    bonds = np.array(dim + nn, dtype=np.int32)
    Jb = np.array([J] * len(dim) + [Jp] * len(nn), dtype=np.float64)
    return bonds, Jb, np.array(dim, dtype=np.int32)


def torus_translations(Lx: int, Ly: int) -> np.ndarray:
    """perms[a + Lx*b][i] = site of (x+a, y+b) for i = (x, y)."""
    out = []
    for b in range(Ly):
        for a in range(Lx):
            out.append([((i % Lx + a) % Lx) + Lx * ((i // Lx + b) % Ly) for i in range(Lx * Ly)])
    return np.array(out, dtype=np.int32)


def chain_characters(N: int, m: int) -> np.ndarray:
    """chi_k(T^n) = exp(i k n) with k = 2 pi m / N (Sec. 3.9.2)."""
    k = 2 * math.pi * m / N
    return np.array([cmath.exp(1j * k * n) for n in range(N)], dtype=np.complex128)


def torus_characters(Lx: int, Ly: int, mx: int, my: int) -> np.ndarray:
    """chi(T_x^a T_y^b) = exp(i (kx a + ky b)), kx = 2 pi mx / Lx, ky = 2 pi my / Ly."""
    kx, ky = 2 * math.pi * mx / Lx, 2 * math.pi * my / Ly
    out = []
    for b in range(Ly):
        for a in range(Lx):
            z = cmath.exp(1j * (kx * a + ky * b))
            out.append(complex(round(z.real, 15), round(z.imag, 15)))
    return np.array(out, dtype=np.complex128)


# ------------------------------------------------------------- workloads
def batched_instances(count: int = 64, seed: int = 4, sizes=(18, 20, 22, 24, 26, 28)):
    """Uneven batch of Heisenberg instances: N uniform over `sizes`, type
    uniform over {chain, ladder (N/2 rungs, each rung twice)}, couplings
    U[0.5, 1.5).  Returns a list of dicts with N, nup=N/2, kind, bonds, J."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        N = int(rng.choice(sizes))
        kind = "chain" if rng.integers(0, 2) == 0 else "ladder"
        bonds = chain(N) if kind == "chain" else ladder(N // 2, 2)
        J = rng.uniform(0.5, 1.5, size=bonds.shape[0]).astype(np.float64)
        out.append(dict(N=N, nup=N // 2, kind=kind, bonds=bonds, J=J))
    return out


# ------------------------------------------------------------ keyed values
# A vector of a block too large to list on the host is generated from the
# block's own state words: with k = SplitMix64(seed), the value of word w is
#   2 u - 1,  u = (SplitMix64(k + (2w + part) gamma) >> 11) 2^-53,
# part 0 the real and part 1 the imaginary part (uniform in [-1, 1),
# exactly representable, so every implementation of this definition gives
# the same bits).  SplitMix64(z) is the generator's output for state z + gamma.
GAMMA = 0x9E3779B97F4A7C15
_M1, _M2 = 0xBF58476D1CE4E5B9, 0x94D049BB133111EB


def _splitmix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z + np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def keyed_values(seed: int, words, cplx: bool = False) -> np.ndarray:
    """Keyed values of the words (numpy, uint64 arithmetic)."""
    w = np.asarray(words, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k = _splitmix64_np(np.array([seed], dtype=np.uint64))[0]

        def part(p):
            z = _splitmix64_np(k + (np.uint64(2) * w + np.uint64(p)) * np.uint64(GAMMA))
            return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53) - 1.0
        re = part(0)
        return re + 1j * part(1) if cplx else re


def _i64(c: int) -> int:
    return c - (1 << 64) if c >= 1 << 63 else c


def keyed_values_torch(seed: int, words, cplx: bool = False):
    """The same values from a torch int64 tensor of words (any device): the
    arithmetic wraps modulo 2^64 and right shifts are made logical by masks."""
    import torch

    def srl(z, s):
        return (z >> s) & ((1 << (64 - s)) - 1)

    def sm(z):
        z = z + _i64(GAMMA)
        z = (z ^ srl(z, 30)) * _i64(_M1)
        z = (z ^ srl(z, 27)) * _i64(_M2)
        return z ^ srl(z, 31)

    k = int(keyed_seed_state(seed))
    w = words.to(torch.int64)

    def part(p):
        z = sm(_i64(k) + (2 * w + p) * _i64(GAMMA))
        return 2.0 * (srl(z, 11).to(torch.float64) * 2.0 ** -53) - 1.0
    re = part(0)
    return torch.complex(re, part(1)) if cplx else re


def keyed_seed_state(seed: int) -> int:
    """k = SplitMix64(seed) as a Python integer."""
    return int(_splitmix64_np(np.array([seed], dtype=np.uint64))[0])

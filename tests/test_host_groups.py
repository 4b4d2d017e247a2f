"""The library's host-side bond-orbit and coupling-invariance helpers
(csrc/xd_groups.h, plain C++) compiled alone with g++ and checked against a
brute-force Python reading of the same definitions."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2505_02901_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_02901_gb300", "csrc")


@pytest.fixture(scope="module")
def shim():
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, f"libhostgroups.{os.getpid()}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", so,
                           os.path.join(HERE, "host_groups_shim.cpp")])
    lib = ctypes.CDLL(so)
    os.remove(so)
    P = ctypes.POINTER
    lib.shim_bond_orbits.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                                     P(ctypes.c_int32)]
    lib.shim_couplings_invariant.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                             ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_int)]
    return lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def brute_orbits(perms, bonds):
    """Orbit ids by the definition: bond p joins the orbit of the first bond q
    whose site pair some g maps onto p's."""
    pair = [frozenset((int(i), int(j))) for i, j in bonds]
    orb, n = [-1] * len(bonds), 0
    for q in range(len(bonds)):
        if orb[q] >= 0:
            continue
        images = {frozenset((int(g[i]), int(g[j]))) for g in perms for i, j in [tuple(bonds[q])]}
        for p in range(len(bonds)):
            if orb[p] < 0 and pair[p] in images:
                orb[p] = n
        n += 1
    return orb, n


def brute_invariant(perms, bonds, J):
    pairs = {}
    for k, (i, j) in enumerate(bonds):
        pairs.setdefault(frozenset((int(i), int(j))), []).append(k)
    for g, row in enumerate(perms):
        for k, (i, j) in enumerate(bonds):
            hit = pairs.get(frozenset((int(row[i]), int(row[j]))), [])
            if not any(J[q] == J[k] for q in hit):
                return 0, g, k
    return 1, 0, 0


CASES = [
    ("square 4x4 space group, J1-J2", W.space_group(4, 4, "square"), W.square_j1j2(4, 4)[0]),
    ("triangular 3x3 space group", W.space_group(3, 3, "triangular"), W.triangular(3)[0]),
    ("6x6 translations, J1-J2", W.torus_translations(6, 6), W.square_j1j2(6, 6)[0]),
    ("D_12 on the J1-J2 chain", W.chain_dihedral(12), W.chain_j1j2(12)[0]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_orbits_and_invariance_match_brute_force(shim, case):
    name, perms, bonds = CASES[case]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    G, N = perms.shape
    nb = len(bonds)
    orb = np.empty(nb, dtype=np.int32)
    n = shim.shim_bond_orbits(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), nb, _p(orb, ctypes.c_int32))
    ob, nbf = brute_orbits(perms, bonds)
    assert n == nbf and orb.tolist() == ob, name
    # couplings constant on each orbit are invariant; breaking one bond is caught
    rng = np.random.default_rng(case)
    per_orbit = rng.uniform(0.5, 1.5, n)
    for J in (per_orbit[orb], np.where(np.arange(nb) == nb // 2, 7.0, per_orbit[orb])):
        J = np.ascontiguousarray(J, dtype=np.float64)
        bg, bk = ctypes.c_int(-1), ctypes.c_int(-1)
        ok = shim.shim_couplings_invariant(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), nb,
                                           _p(J, ctypes.c_double), ctypes.byref(bg), ctypes.byref(bk))
        want = brute_invariant(perms, bonds, J)
        assert (ok, bg.value if not ok else 0, bk.value if not ok else 0) == want, name


def test_duplicated_bonds(shim):
    """A ladder that lists every rung twice under its leg translations: the
    legs are two orbits and all rung copies a third; the two copies of a rung
    may carry different couplings as long as every rung carries both."""
    L = 8
    bonds = np.ascontiguousarray(W.ladder(L, 2), dtype=np.int32)
    N = 2 * L
    perms = np.ascontiguousarray([[((i % L + n) % L) + L * (i // L) for i in range(N)] for n in range(L)],
                                 dtype=np.int32)
    orb = np.empty(len(bonds), dtype=np.int32)
    n = shim.shim_bond_orbits(N, L, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds),
                              _p(orb, ctypes.c_int32))
    ob, nbf = brute_orbits(perms, bonds)
    assert n == nbf == 3 and orb.tolist() == ob  # leg 0, leg 1, both rung copies
    J = np.ones(len(bonds))
    J[2 * L:3 * L], J[3 * L:] = 0.7, 1.3  # copy A and copy B of every rung
    J = np.ascontiguousarray(J)
    bg, bk = ctypes.c_int(), ctypes.c_int()
    assert shim.shim_couplings_invariant(N, L, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds),
                                         _p(J, ctypes.c_double), ctypes.byref(bg), ctypes.byref(bk)) == 1
    J[3 * L] = 0.7  # one rung now has 0.7 twice: the image of copy B (1.3) is missing there
    assert shim.shim_couplings_invariant(N, L, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds),
                                         _p(J, ctypes.c_double), ctypes.byref(bg), ctypes.byref(bk)) == 0
    assert brute_invariant(perms, bonds, J) == (0, bg.value, bk.value)


def _act(perm, s):
    """(g s)_i = s_{g(i)} on a state word."""
    return sum(((s >> int(perm[i])) & 1) << i for i in range(len(perm)))


def _tables(shim, perms, bonds):
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    G, N = perms.shape
    nb = len(bonds)
    nchunk = (N + 7) // 8
    meta = np.zeros(6, dtype=np.int32)
    act = np.zeros(G * nchunk * 256, dtype=np.uint64)
    minrot, amask = np.zeros(256, dtype=np.uint8), np.zeros(256, dtype=np.uint8)
    tg, tpp = np.full(G, -1, dtype=np.int16), np.full(G, -1, dtype=np.int16)
    pm = np.zeros(max(1, G * nb), dtype=np.uint64)
    cg = np.full(2 * N, -1, dtype=np.int16)
    P = ctypes.POINTER
    shim.shim_group_tables.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                                       P(ctypes.c_int32), P(ctypes.c_uint64), P(ctypes.c_uint8), P(ctypes.c_uint8),
                                       P(ctypes.c_int16), P(ctypes.c_int16), P(ctypes.c_uint64), P(ctypes.c_int16)]
    shim.shim_group_tables(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), nb, _p(meta, ctypes.c_int32),
                           _p(act, ctypes.c_uint64), _p(minrot, ctypes.c_uint8), _p(amask, ctypes.c_uint8),
                           _p(tg, ctypes.c_int16), _p(tpp, ctypes.c_int16), _p(pm, ctypes.c_uint64),
                           _p(cg, ctypes.c_int16))
    return perms, bonds, dict(zip(("nchunk", "tx", "ty", "tnp", "cn", "cdih"), meta.tolist())), act, minrot, amask, \
        tg, tpp, pm, cg


GROUPS = [
    # name, perms, bonds, expected (tx, ty, cosets or 0, ring cn, cdih)
    ("square 4x4 space group", W.space_group(4, 4, "square"), W.square_j1j2(4, 4)[0], (4, 4, 8, 0, 0)),
    ("triangular 3x3 space group", W.space_group(3, 3, "triangular"), W.triangular(3)[0], (3, 3, 12, 0, 0)),
    ("rectangular 4x6 space group", W.space_group(4, 6, "rectangular"), W.square_j1j2(4, 6)[0], (4, 6, 4, 0, 0)),
    ("6x6 translations", W.torus_translations(6, 6), W.square_j1j2(6, 6)[0], (6, 6, 0, 0, 0)),
    ("D_8 (one-row torus)", W.chain_dihedral(8), W.chain(8), (8, 1, 2, 0, 0)),
    ("D_12 (ring)", W.chain_dihedral(12), W.chain_j1j2(12)[0], (0, 0, 0, 12, 1)),
    ("C_12 (ring)", W.chain_translations(12), W.chain(12), (0, 0, 0, 12, 0)),
    ("C4v alone on 4x4 (no translations)", W.space_group(4, 4, "square")[::16], W.square_j1j2(4, 4)[0],
     (0, 0, 0, 0, 0)),
]


@pytest.mark.parametrize("case", range(len(GROUPS)))
def test_group_tables(shim, case):
    name, perms, bonds, want = GROUPS[case]
    rng = np.random.default_rng(case)
    perms = np.asarray(perms)
    scramble = rng.permutation(len(perms))  # any element order
    scramble = np.r_[scramble[scramble == 0], scramble[scramble != 0]] if case % 2 else scramble
    perms, bonds, m, act, minrot, amask, tg, tpp, pm, cg = _tables(shim, perms[scramble], bonds)
    G, N = perms.shape
    assert (m["tx"], m["ty"], m["tnp"], m["cn"], m["cdih"]) == want, name
    # byte tables of the action
    for _ in range(20):
        s = int(rng.integers(0, 1 << N))
        for g in rng.integers(0, G, 3):
            got = 0
            for c in range(m["nchunk"]):
                got |= int(act[(int(g) * m["nchunk"] + c) * 256 + ((s >> (8 * c)) & 255)])
            assert got == _act(perms[g], s)
    if m["tx"]:
        Lx, Ly = m["tx"], m["ty"]
        ncos = max(1, m["tnp"])
        assert (perms[tpp[0]] == np.arange(N)).all()  # p_0 is the identity
        assert sorted(tg[:ncos * N].tolist()) == list(range(G))  # every element once
        for k in range(ncos):
            for t in range(N):
                a, b = t % Lx, t // Lx
                tr = [((i % Lx + a) % Lx) + Lx * ((i // Lx + b) % Ly) for i in range(N)]
                assert perms[tg[k * N + t]].tolist() == [int(perms[tpp[k]][tr[i]]) for i in range(N)]
        for r in range(1 << Lx):
            rots = [((r >> a) | (r << (Lx - a))) & ((1 << Lx) - 1) for a in range(Lx)]
            assert minrot[r] == min(rots)
            assert amask[r] == sum(1 << a for a in range(Lx) if rots[a] == min(rots))
        for k in range(1, m["tnp"]):
            for q, (i, j) in enumerate(bonds):
                assert int(pm[(k - 1) * len(bonds) + q]) == _act(perms[tpp[k]], (1 << int(i)) | (1 << int(j)))
    if m["cn"]:
        for n in range(N):
            assert perms[cg[n]].tolist() == [(i + n) % N for i in range(N)]
            if m["cdih"]:
                assert perms[cg[N + n]].tolist() == [(n - i) % N for i in range(N)]


def _brute_rep(perms, words):
    """Smallest image over every group element, |Stab|, by the definition
    (g s)_i = s_{g(i)}."""
    G, N = perms.shape
    bits = ((words[:, None] >> np.arange(N, dtype=np.uint64)) & np.uint64(1)).astype(np.uint64)
    img = np.zeros((len(words), G), dtype=np.uint64)
    for g in range(G):
        img[:, g] = (bits[:, perms[g]] << np.arange(N, dtype=np.uint64)).sum(axis=1, dtype=np.uint64)
    rep = img.min(axis=1)
    return rep, (img == rep[:, None]).sum(axis=1), img


def _apply_perm(perm, w):
    N = len(perm)
    return sum(((int(w) >> int(perm[i])) & 1) << i for i in range(N))


TORUS_CASES = [
    ("6x6 translations", W.torus_translations(6, 6), W.square_j1j2(6, 6)[0], 18),
    ("6x6 square space group", W.space_group(6, 6, "square"), W.square_j1j2(6, 6)[0], 18),
    ("6x6 triangular space group", W.space_group(6, 6, "triangular"), W.triangular(6)[0], 17),
    ("4x4 square space group", W.space_group(4, 4, "square"), W.square_j1j2(4, 4)[0], 8),
    ("8x8 translations", W.torus_translations(8, 8), W.square_j1j2(8, 8)[0], 32),
    ("3x5 translations", W.torus_translations(3, 5), W.square_j1j2(3, 5)[0], 7),
]


@pytest.mark.parametrize("use_cut", [0, 1])
@pytest.mark.parametrize("case", range(len(TORUS_CASES)))
def test_torus_narrowing_search_matches_every_element(shim, case, use_cut):
    """The row-by-row narrowing search (xd_orbit.h) returns the smallest image
    over every group element, the stabiliser size, and an element reaching
    it, on random words, periodic words (many equal candidates) and the
    all-zero / all-one words."""
    name, perms, bonds, nup = TORUS_CASES[case]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    G, N = perms.shape
    rng = np.random.default_rng(11 + case)
    words = []
    for _ in range(3000):
        sites = rng.choice(N, size=int(rng.integers(0, N + 1)) if _ % 3 == 0 else nup, replace=False)
        words.append(sum(1 << int(i) for i in sites))
    # words invariant under translations: stripes and checkerboards of the torus
    Lx = {"6x6": 6, "4x4": 4, "8x8": 8, "3x5": 3}[name.split()[0]]
    Ly = N // Lx
    for pat in (0b01, 0b011, 0b0101, 0b0011):
        row = sum(((pat >> (x % 4)) & 1) << x for x in range(Lx))
        words.append(sum(row << (Lx * y) for y in range(Ly)))
        words.append(sum((row if y % 2 else (~row & ((1 << Lx) - 1))) << (Lx * y) for y in range(Ly)))
    words += [0, (1 << N) - 1]
    words = np.array(words, dtype=np.uint64)
    n = len(words)
    rep = np.zeros(n, np.uint64)
    cnt = np.zeros(n, np.int32)
    u = np.zeros(n, np.int32)
    P = ctypes.POINTER
    shim.shim_torus_orbit.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                                      ctypes.c_int64, P(ctypes.c_uint64), P(ctypes.c_uint64), P(ctypes.c_int32),
                                      P(ctypes.c_int32), ctypes.c_int]
    ok = shim.shim_torus_orbit(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds), n,
                               _p(words, ctypes.c_uint64), _p(rep, ctypes.c_uint64), _p(cnt, ctypes.c_int32),
                               _p(u, ctypes.c_int32), use_cut)
    if use_cut and Lx > 7:
        assert ok == 0  # no cut table for rows of 8 sites
        return
    assert ok == 1, name
    brep, bcnt, img = _brute_rep(perms, words)
    np.testing.assert_array_equal(rep, brep)
    np.testing.assert_array_equal(cnt, bcnt)
    np.testing.assert_array_equal(img[np.arange(n), u], brep)
    assert bcnt.max() > 1  # the periodic words exercise equal candidates


@pytest.mark.parametrize("case", range(len(TORUS_CASES)))
def test_torus_incremental_top_step(shim, case):
    """The top step from a row state refreshed in the two flipped rows
    (byte-wise minimum and comparison) equals the top step computed from the
    flipped word, for random words and site pairs, zero and full words."""
    name, perms, bonds, nup = TORUS_CASES[case]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    G, N = perms.shape
    rng = np.random.default_rng(3 + case)
    n = 20000
    words = np.array([sum(1 << int(i) for i in rng.choice(N, size=int(rng.integers(0, N + 1)), replace=False))
                      for _ in range(n)] + [0, (1 << N) - 1], dtype=np.uint64)
    ij = np.ascontiguousarray(np.stack([rng.choice(N, 2, replace=False) for _ in range(len(words))]), dtype=np.int32)
    P = ctypes.POINTER
    shim.shim_top_rows_mismatch.restype = ctypes.c_int64
    shim.shim_top_rows_mismatch.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                            ctypes.c_int, ctypes.c_int64, P(ctypes.c_uint64), P(ctypes.c_int32)]
    bad = shim.shim_top_rows_mismatch(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds),
                                      len(words), _p(words, ctypes.c_uint64), _p(ij, ctypes.c_int32))
    if name.startswith("8x8"):
        assert bad == -2  # rows of 8 sites take the search from the word
        return
    assert bad == 0, name


@pytest.mark.parametrize("case", range(len(TORUS_CASES)))
def test_torus_top_step_from_three_smallest_rows(shim, case):
    """The top step of a flipped word from the three smallest rows of the
    word before the flip (the rows it leaves untouched) and the two new rows
    equals the top step computed from the flipped word: random words, zero
    and full words, random site pairs (same row and different rows)."""
    name, perms, bonds, nup = TORUS_CASES[case]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    G, N = perms.shape
    rng = np.random.default_rng(13 + case)
    n = 20000
    words = np.array([sum(1 << int(i) for i in rng.choice(N, size=int(rng.integers(0, N + 1)), replace=False))
                      for _ in range(n)] + [0, (1 << N) - 1], dtype=np.uint64)
    ij = np.ascontiguousarray(np.stack([rng.choice(N, 2, replace=False) for _ in range(len(words))]), dtype=np.int32)
    P = ctypes.POINTER
    shim.shim_top3_mismatch.restype = ctypes.c_int64
    shim.shim_top3_mismatch.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int32),
                                        ctypes.c_int, ctypes.c_int64, P(ctypes.c_uint64), P(ctypes.c_int32)]
    bad = shim.shim_top3_mismatch(N, G, _p(perms, ctypes.c_int32), _p(bonds, ctypes.c_int32), len(bonds),
                                  len(words), _p(words, ctypes.c_uint64), _p(ij, ctypes.c_int32))
    if name.startswith("8x8"):
        assert bad == -2
        return
    assert bad == 0, name

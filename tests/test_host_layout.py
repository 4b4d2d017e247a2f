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
    L.shim_ordered_items.restype = ctypes.c_longlong
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


def _arr(fn, ctype, n):
    fn.restype = ctypes.POINTER(ctype)
    return np.ctypeslib.as_array(fn(), shape=(max(1, n),))[:n].copy() if n else np.zeros(0)


def block_product_twin(lay, N, nup, bonds, J, x, L_at=0):
    """y = H x read off the block tables the way the FP64 block kernel uses
    them: per prefix block h, postfix flips through ptab (the zero slot for
    "no flip"), prefix flips as whole neighbour blocks at the same position,
    cross flips through xtab from the neighbour block of the flipped prefix
    bit with J/2 (x_target - x_row), and the diagonal J_cross/4 + prefix
    and postfix terms."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    sz = (ctypes.c_int * 9)()
    lay.shim_block_build_at(N, nup, L_at, bonds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(bonds), sz)
    L, npost, npre, ncross, ncsite, nslot, npost_pad, maxblk, norder = list(sz)
    P, nlo = N - L, 1 << L
    hi_off = _arr(lay.shim_hi_off, ctypes.c_int64, (1 << P) + 1)
    lo_list = _arr(lay.shim_lo_list, ctypes.c_uint32, nlo)
    lo_off = _arr(lay.shim_lo_off, ctypes.c_uint32, L + 2)
    post = _arr(lay.shim_post, ctypes.c_int32, npost)
    pre = _arr(lay.shim_pre, ctypes.c_int32, 3 * npre).reshape(-1, 3)
    cross = _arr(lay.shim_cross, ctypes.c_int32, 4 * ncross).reshape(-1, 4)
    csite = _arr(lay.shim_csite, ctypes.c_int32, 3 * ncsite).reshape(-1, 3)
    ptab = _arr(lay.shim_ptab, ctypes.c_uint16, npost_pad * nlo).reshape(npost_pad, nlo).astype(np.int64)
    xtab = _arr(lay.shim_xtab, ctypes.c_uint16, nslot * nlo).reshape(nslot, nlo).astype(np.int64)
    order = _arr(lay.shim_order, ctypes.c_uint32, norder)
    # postfix diagonal per class position (the kernel's dpost table)
    dpost = np.zeros(nlo)
    for k in post:
        i, j = bonds[k]
        dpost += np.where(((lo_list >> i) & 1) == ((lo_list >> j) & 1), 0.25, -0.25) * J[k]
    jcross = 0.25 * sum(J[c[2]] for c in cross)
    pc = np.zeros(npost_pad)
    pc[:npost] = 0.5 * J[post]
    y = np.zeros_like(x)
    for h in order.tolist():
        m = nup - bin(h).count("1")
        l0, n, off = int(lo_off[m]), int(lo_off[m + 1] - lo_off[m]), int(hi_off[h])
        xs = np.zeros(maxblk + 1)
        xs[:n] = x[off:off + n]
        g = l0 + np.arange(n)
        acc = (pc[:, None] * xs[ptab[:, g]]).sum(axis=0)
        dpre = 0.0
        for a, b, k in pre:
            if ((h >> a) & 1) != ((h >> b) & 1):
                dpre -= 0.25 * J[k]
                o2 = int(hi_off[h ^ (1 << a) ^ (1 << b)])
                acc += 0.5 * J[k] * x[o2:o2 + n]
            else:
                dpre += 0.25 * J[k]
        l = lo_list[g]
        for a, q0, q1 in csite:
            hb = (h >> a) & 1
            o2 = int(hi_off[h ^ (1 << a)])
            for q in range(q0, q1):
                site, k, slot = cross[q][1], cross[q][2], cross[q][3]
                f = ((l >> site) & 1) == (1 - hb)
                tgt = np.where(f, o2 + xtab[slot, g], 0)  # read only where the bond flips
                acc += np.where(f, 0.5 * J[k] * (x[tgt] - xs[:n]), 0.0)
        y[off:off + n] = (dpre + jcross + dpost[g]) * xs[:n] + acc
    return y


@pytest.mark.parametrize("case", range(5))
def test_block_tables_reproduce_the_product(lay, orc, case):
    from paper_2505_02901_gb300 import workloads as W
    rng = np.random.default_rng(case)
    if case == 0:
        N, nup, bonds = 20, 10, W.random_bonds(20, 45, 3)
    elif case == 1:
        N, nup, bonds = 20, 10, W.square_j1j2(4, 5)[0]
    elif case == 2:
        N, nup, bonds = 20, 9, W.ladder(10, 2)
    elif case == 3:
        N, nup, bonds = 22, 11, W.chain(22)
    else:
        N, nup, bonds = 24, 4, W.random_bonds(24, 60, 8)
    J = rng.uniform(0.5, 1.5, len(bonds))
    st = orc.enumerate_states(N, nup)
    x = rng.standard_normal(st.size)
    y = block_product_twin(lay, N, nup, bonds, J, x)
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("N,nup", [(24, 12), (26, 7)])
def test_tables_at_the_batched_width(lay, orc, N, nup):
    """The FP32 batched product keeps a postfix of L = min(12, N - 12) bits;
    its tables (same construction at that L) reproduce the product."""
    from paper_2505_02901_gb300 import workloads as W
    bonds = W.square_j1j2(4, N // 4)[0] if N % 4 == 0 else W.random_bonds(N, 2 * N, 5)
    rng = np.random.default_rng(N)
    J = rng.uniform(0.5, 1.5, len(bonds))
    st = orc.enumerate_states(N, nup)
    x = rng.standard_normal(st.size)
    y = block_product_twin(lay, N, nup, bonds, J, x, L_at=min(12, N - 12))
    yo = orc.apply_u1(N, st, bonds, J, x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("N,nup", [(24, 12), (28, 14), (30, 3), (26, 20)])
def test_work_items(lay, N, nup):
    """Every prefix with a non-empty block appears in exactly one item; an
    item holds kB prefixes of one class, ascending, padded only at its end."""
    L = min(12, N - 12)
    P, kB, empty = N - L, 8, 0xFFFFFFFF
    lay.shim_items.restype = ctypes.c_longlong
    lay.shim_items.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_longlong]
    n = lay.shim_items(P, nup, L, kB, empty, None, 0)
    out = np.zeros(n, dtype=np.uint32)
    assert lay.shim_items(P, nup, L, kB, empty, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n) == n
    assert n % kB == 0
    want = [h for h in range(1 << P) if 0 <= nup - bin(h).count("1") <= L]
    got = [int(h) for h in out if h != empty]
    assert sorted(got) == want
    last = {}
    for it in out.reshape(-1, kB):
        real = [int(h) for h in it if h != empty]
        assert real and all(h == empty for h in it[len(real):])  # padding at the end only
        cls = {nup - bin(h).count("1") for h in real}
        assert len(cls) == 1
        m = cls.pop()
        assert real == sorted(real) and real[0] > last.get(m, -1)
        last[m] = real[-1]


def _passes(lay, P, pre, W, maxp=3):
    pre = np.ascontiguousarray(np.asarray(pre, dtype=np.int32).reshape(-1))
    n = lay.shim_choose_passes(P, pre.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(pre) // 3, W, maxp)
    out = []
    for p in range(n):
        low = np.zeros(64, dtype=np.int32)
        bd = np.zeros(len(pre) // 3 + 1, dtype=np.int32)
        nl = lay.shim_pass_low(p, low.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        nbd = lay.shim_pass_bonds(p, bd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        out.append((list(low[:nl]), list(bd[:nbd])))
    return out


def _prefix_triples(N, L, bonds):
    return [(min(i, j) - L, max(i, j) - L, k) for k, (i, j) in enumerate(bonds) if min(i, j) >= L]


@pytest.mark.parametrize("lattice,W,npass", [((4, 8), 12, 2), ((6, 6), 12, 3), ((6, 6), 18, 2), ((4, 7), 12, 2), ((4, 7), 16, 1), ((4, 8), 20, 1)])
def test_prefix_passes_cover_every_bond_locally(lay, lattice, W, npass):
    """Every prefix bond lands in exactly one pass; on the J1-J2 tori each
    pass's bonds have both bits in its window of at most W bits (whole rows:
    two passes for the 4x8 prefix of 5 rows of 4 sites, three for the 6x6
    prefix of 4 rows of 6 at W = 12)."""
    from paper_2505_02901_gb300 import workloads as W_
    Lx, Ly = lattice
    N = Lx * Ly
    L = 12
    bonds, _ = W_.square_j1j2(Lx, Ly)
    pre = _prefix_triples(N, L, bonds)
    P = N - L
    passes = _passes(lay, P, [t for tr in pre for t in tr], W)
    assert len(passes) == npass
    seen = sorted(q for _, bd in passes for q in bd)
    assert seen == list(range(len(pre)))
    for low, bd in passes:
        assert len(low) <= W and low == sorted(low)
        for q in bd:
            a, c, _ = pre[q]
            assert a in low and c in low


def test_prefix_passes_random_graph_and_limits(lay):
    """Any bond graph: every bond assigned once, at most max_passes passes;
    a graph that fits one window takes one pass."""
    rng = np.random.default_rng(0)
    P = 22
    pre = []
    for k in range(90):
        a, c = rng.choice(P, 2, replace=False)
        pre.append((min(a, c), max(a, c), k))
    for maxp in (1, 2, 3):
        passes = _passes(lay, P, [t for tr in pre for t in tr], 10, maxp)
        assert 1 <= len(passes) <= maxp
        assert sorted(q for _, bd in passes for q in bd) == list(range(len(pre)))
    passes = _passes(lay, 8, [0, 1, 0, 2, 7, 1], 8)
    assert len(passes) == 1 and sorted(passes[0][1]) == [0, 1]


def test_ordered_items_cover_every_block_once(lay):
    """Items of kB same-class prefixes in key order: every non-empty prefix
    exactly once, one class per item, padding only at the end of a class."""
    P, nup, L, kB = 12, 10, 8, 4
    low = np.array([10, 11, 0, 1], dtype=np.int32)
    cap = 1 << 16
    out = np.zeros(cap, dtype=np.uint32)
    n = lay.shim_ordered_items(P, nup, L, kB, 0xffffffff, low.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               len(low), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap)
    items = out[:n].reshape(-1, kB)
    real = items[items != 0xffffffff]
    want = [h for h in range(1 << P) if 0 <= nup - bin(h).count("1") <= L]
    assert sorted(real.tolist()) == want
    for it in items:
        cls = {bin(int(h)).count("1") for h in it if h != 0xffffffff}
        assert len(cls) == 1

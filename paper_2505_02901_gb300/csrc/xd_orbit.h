// xd_orbit.h -- the representative of a word under a group holding the
// translations of an Lx x Ly torus (Sec. 3.10: the representative of an
// orbit is its smallest image), for host and device code.
//
// The group is the union of the cosets {s -> T_{a,b}(p_k s)} (p_0 the
// identity; T alone when there is one coset).  (T_{a,b} w) puts in row y the
// row (y + b) mod Ly of w rotated by a (new bit x = old bit (x + a) mod Lx);
// row Ly - 1 holds the most significant bits.  The smallest image of w over
// T therefore has as top row the smallest rotation of any row of w, and is
// found row by row from the top: a candidate set of translations (a, b) is
// cut, row by row, to those reaching the smallest value of that row.  Once
// one candidate is left its image is formed in one go.  Across cosets the
// running smallest image bounds the search: a coset whose partial image
// exceeds it stops.
//
// Candidates are the bits a + 8 b of a 64-bit word (Lx <= 8, Ly <= 8).
// Tables: rowtab[r] = smallest rotation of the Lx-bit row r (low byte) and
// the mask of the rotations a reaching it (high byte); cut[(r << Lx) | A]
// (Lx <= 7, optional) = the smallest rot_a(r) over a in the mask A (low byte)
// and the a in A reaching it (high byte), so that one row step of a
// candidate b costs one lookup however many rotations it still holds.

#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define XD_HD __host__ __device__ __forceinline__
#else
#define XD_HD inline
#endif

namespace xd {

XD_HD int orb_ctz(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __ffsll((long long)v) - 1;
#else
    return __builtin_ctzll(v);
#endif
}

XD_HD int orb_popc(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __popcll(v);
#else
    return __builtin_popcountll(v);
#endif
}

struct TorusGeo {
    int Lx, Ly, N;
    uint32_t rowmask;       // 2^Lx - 1
    uint64_t nmask;         // 2^N - 1
    uint64_t rep1;          // bit 0 of every row
    const uint16_t *rowtab; // [2^Lx]
    const uint16_t *cut;    // [2^(2 Lx)] or null
};

XD_HD TorusGeo torus_geo(int Lx, int Ly, const uint16_t *rowtab, const uint16_t *cut = nullptr) {
    TorusGeo g;
    g.Lx = Lx;
    g.Ly = Ly;
    g.N = Lx * Ly;
    g.rowmask = (1u << Lx) - 1;
    g.nmask = ~0ull >> (64 - g.N);
    g.rep1 = 0;
    for (int y = 0; y < Ly; ++y) g.rep1 |= 1ull << (Lx * y);
    g.rowtab = rowtab;
    g.cut = cut;
    return g;
}

XD_HD uint32_t torus_row(const TorusGeo &g, uint64_t w, int y) {
    return (uint32_t)(w >> (g.Lx * y)) & g.rowmask;
}

// T_{a,b} w on the whole word: the rows move down by b, every row rotates by a.
XD_HD uint64_t torus_translate(const TorusGeo &g, uint64_t w, int a, int b) {
    const int sb = g.Lx * b;  // every shift below stays under 64
    w = ((w >> sb) | (w << ((g.N - sb) & 63))) & g.nmask;
    const uint64_t low = g.rep1 * ((1ull << (g.Lx - a)) - 1);  // bits that move down by a
    return ((w >> a) & low) | ((w << (g.Lx - a)) & (g.nmask ^ low));
}

// Smallest top row over the translations of w (*top) and the candidates
// reaching it: the row y that comes to the top under T_{a,b} has b = (y + 1) mod Ly.
XD_HD uint64_t torus_top(const TorusGeo &g, uint64_t w, uint32_t *top) {
    uint32_t best = 0xffffffffu;
    uint64_t M = 0;
    for (int y = 0; y < g.Ly; ++y) {
        const uint32_t e = g.rowtab[torus_row(g, w, y)];
        const uint32_t v = e & 0xffu;
        const int b = y + 1 == g.Ly ? 0 : y + 1;
        const uint64_t bits = (uint64_t)(e >> 8) << (8 * b);
        if (v < best) {
            best = v;
            M = bits;
        } else if (v == best) {
            M |= bits;
        }
    }
    *top = best;
    return M;
}

// Narrows the candidates M (all with top row `top`) of w to those reaching the
// smallest image *img.  With bounded set the search stops, returning false,
// as soon as the image is known to exceed bound.
XD_HD bool torus_narrow(const TorusGeo &g, uint64_t w, uint32_t top, uint64_t &M, bool bounded,
                        uint64_t bound, uint64_t *img_out) {
    const int ytop = g.Ly - 1;
    uint64_t img = (uint64_t)top << (g.Lx * ytop);
    bool tight = bounded && torus_row(g, bound, ytop) == top;  // image prefix == bound prefix
    for (int y = ytop - 1; y >= 0; --y) {
        if ((M & (M - 1)) == 0) {  // one candidate: its image in one go (the identity: w)
            const int q = orb_ctz(M);
            *img_out = q ? torus_translate(g, w, q & 7, q >> 3) : w;
            return !(tight && *img_out > bound);
        }
        uint32_t vmin = 0xffffffffu;
        uint64_t M2 = 0, bm = M;
        while (bm) {
            const int b = orb_ctz(bm) >> 3;
            uint32_t am = (uint32_t)(bm >> (8 * b)) & 0xffu;
            bm &= ~(0xffull << (8 * b));
            int ys = y + b;
            if (ys >= g.Ly) ys -= g.Ly;
            const uint32_t r = torus_row(g, w, ys);
            uint32_t v, sub;
            if (g.cut) {
                const uint32_t e = g.cut[(r << g.Lx) | am];
                v = e & 0xffu;
                sub = e >> 8;
            } else {
                v = 0xffffffffu;
                sub = 0;
                while (am) {
                    const int a = orb_ctz(am);
                    am &= am - 1;
                    const uint32_t va = a ? (((r >> a) | (r << (g.Lx - a))) & g.rowmask) : r;
                    if (va < v) {
                        v = va;
                        sub = 1u << a;
                    } else if (va == v) {
                        sub |= 1u << a;
                    }
                }
            }
            const uint64_t bits = (uint64_t)sub << (8 * b);
            if (v < vmin) {
                vmin = v;
                M2 = bits;
            } else if (v == vmin) {
                M2 |= bits;
            }
        }
        M = M2;
        img |= (uint64_t)vmin << (g.Lx * y);
        if (tight) {
            const uint32_t br = torus_row(g, bound, y);
            if (vmin > br) return false;
            tight = vmin == br;
        }
    }
    *img_out = img;
    return true;
}

// Row state of a word for the top step (rows of at most 7 sites): byte y of
// PM = smallest rotation of row y, byte y of PA = the rotations reaching it
// (bytes y >= Ly: 0x7f / 0, above every row value and never a candidate).
// A flip changes one or two rows; torus_rows_set refreshes row y from the
// flipped word, and torus_top_rows gives what torus_top gives, by byte-wise
// minimum and comparison on plain integer operations (every byte < 128).
XD_HD uint32_t bytes_min4(uint32_t a, uint32_t b) {
    const uint32_t ge = ((a | 0x80808080u) - b) & 0x80808080u;  // 0x80 where a >= b
    const uint32_t sel = (ge >> 7) * 0xffu;
    return (b & sel) | (a & ~sel);
}

XD_HD uint32_t bytes_min8(uint64_t v) {
    uint32_t m = bytes_min4((uint32_t)v, (uint32_t)(v >> 32));
    m = bytes_min4(m, m >> 16);
    m = bytes_min4(m, m >> 8);
    return m & 0xffu;
}

// 0xff in every byte of v equal to the byte t, 0 elsewhere
XD_HD uint32_t bytes_eq4(uint32_t v, uint32_t t) {
    const uint32_t x = v ^ (t * 0x01010101u);  // zero bytes where equal
    const uint32_t z = ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x | 0x7f7f7f7fu);  // 0x80 in zero bytes
    return (z >> 7) * 0xffu;
}

XD_HD uint64_t bytes_eq8(uint64_t v, uint32_t t) {
    return (uint64_t)bytes_eq4((uint32_t)v, t) | ((uint64_t)bytes_eq4((uint32_t)(v >> 32), t) << 32);
}

XD_HD void torus_rows_set(const TorusGeo &g, uint64_t &PM, uint64_t &PA, uint64_t w, int y) {
    const uint32_t e = g.rowtab[torus_row(g, w, y)];
    const uint64_t keep = ~(0xffull << (8 * y));
    PM = (PM & keep) | ((uint64_t)(e & 0xffu) << (8 * y));
    PA = (PA & keep) | ((uint64_t)(e >> 8) << (8 * y));
}

XD_HD void torus_rows(const TorusGeo &g, uint64_t w, uint64_t &PM, uint64_t &PA) {
    PM = 0x7f7f7f7f7f7f7f7full;
    PA = 0;
    for (int y = 0; y < g.Ly; ++y) torus_rows_set(g, PM, PA, w, y);
}

XD_HD uint64_t torus_top_rows(const TorusGeo &g, uint64_t PM, uint64_t PA, uint32_t *top) {
    const uint32_t best = bytes_min8(PM);
    const uint64_t Mr = bytes_eq8(PM, best) & PA;  // byte y: rotations of row y reaching best
    *top = best;
    // row y comes to the top under b = (y + 1) mod Ly
    const int sh = 8 * (g.Ly - 1);
    return ((Mr << 8) | (Mr >> sh)) & (~0ull >> (64 - 8 * g.Ly));
}

// Top step from the three smallest rows of the word (translations alone,
// rows of at most 7 sites).  For a word w, RowTop3 holds the three smallest
// row minima in ascending order (ties kept) with their rows, and for each
// such value the candidates of every row reaching it (bits a + 8 b, b the
// translation bringing the row to the top).  A flip that changes rows y1
// and y2 leaves the others as they were: the smallest of those is the first
// of the three whose row is neither y1 nor y2, and its candidates are those
// of its value with rows y1 and y2 taken out; the two new rows join from the
// row table.  torus_top_flip then gives what torus_top gives on the flipped
// word.
struct RowTop3 {
    uint32_t v;   // bytes 0..2: the three smallest minima (0xff: fewer rows)
    uint32_t y;   // bytes 0..2: their rows
    uint64_t m0, m1, m2;
};

XD_HD uint64_t row_cands(const TorusGeo &g, int y, uint32_t am) {
    return (uint64_t)am << (y + 1 == g.Ly ? 0 : 8 * (y + 1));
}

XD_HD void torus_top3(const TorusGeo &g, uint64_t w, RowTop3 &t) {
    uint32_t v0 = 0xffu, v1 = 0xffu, v2 = 0xffu, y0 = 0, y1 = 0, y2 = 0;
    for (int y = 0; y < g.Ly; ++y) {  // insertion into the three smallest (stable)
        const uint32_t val = g.rowtab[torus_row(g, w, y)] & 0xffu;
        if (val < v0) {
            v2 = v1; y2 = y1; v1 = v0; y1 = y0; v0 = val; y0 = (uint32_t)y;
        } else if (val < v1) {
            v2 = v1; y2 = y1; v1 = val; y1 = (uint32_t)y;
        } else if (val < v2) {
            v2 = val; y2 = (uint32_t)y;
        }
    }
    t.v = v0 | (v1 << 8) | (v2 << 16);
    t.y = y0 | (y1 << 8) | (y2 << 16);
    t.m0 = t.m1 = t.m2 = 0;
    for (int y = 0; y < g.Ly; ++y) {
        const uint32_t e = g.rowtab[torus_row(g, w, y)], val = e & 0xffu;
        const uint64_t c = row_cands(g, y, e >> 8);
        if (val == v0) t.m0 |= c;
        if (val == v1) t.m1 |= c;
        if (val == v2) t.m2 |= c;
    }
}

XD_HD uint64_t torus_top_flip(const TorusGeo &g, const RowTop3 &t, uint64_t w, int y1, int y2, uint32_t *top) {
    // the smallest row left untouched: the first of the three that is neither y1 nor y2
    const int r0 = (int)(t.y & 0xffu), r1 = (int)((t.y >> 8) & 0xffu);
    const bool k0 = r0 != y1 && r0 != y2, k1 = r1 != y1 && r1 != y2;
    const uint32_t ex = k0 ? (t.v & 0xffu) : k1 ? ((t.v >> 8) & 0xffu) : ((t.v >> 16) & 0xffu);
    const uint64_t mx = k0 ? t.m0 : k1 ? t.m1 : t.m2;
    const uint64_t keep = ~row_cands(g, y1, 0xffu) & ~row_cands(g, y2, 0xffu);
    const uint32_t e1 = g.rowtab[torus_row(g, w, y1)], e2 = g.rowtab[torus_row(g, w, y2)];
    const uint32_t v1 = e1 & 0xffu, v2 = e2 & 0xffu;
    uint32_t best = ex < v1 ? ex : v1;
    best = best < v2 ? best : v2;
    uint64_t M = ex == best ? (mx & keep) : 0;
    if (v1 == best) M |= row_cands(g, y1, e1 >> 8);
    if (v2 == best) M |= row_cands(g, y2, e2 >> 8);
    *top = best;
    return M;
}

struct TorusOrbit {
    uint64_t rep;  // smallest image
    int k, q;      // a winning coset and translation (bit q = a + 8 b)
    int cnt;       // number of (coset, translation) pairs reaching rep
};

// Smallest image of s over the union of ncos cosets; wk(k, &w, &top)
// returns p_k s in w, its top row in top and the candidates reaching it.
template <class W>
XD_HD TorusOrbit torus_orbit_top(const TorusGeo &g, int ncos, W wk) {
    TorusOrbit o{~0ull, 0, 0, 0};
    uint32_t gbest = 0xffffffffu;  // top row of o.rep (o.cnt > 0)
    for (int k = 0; k < ncos; ++k) {
        uint64_t w;
        uint32_t top;
        uint64_t M = wk(k, &w, &top);
        if (o.cnt && top > gbest) continue;
        const bool bounded = o.cnt && top == gbest;
        uint64_t img;
        if (!torus_narrow(g, w, top, M, bounded, o.rep, &img)) continue;
        if (!bounded || img < o.rep) {
            o.rep = img;
            o.k = k;
            o.q = orb_ctz(M);
            o.cnt = orb_popc(M);
            gbest = top;
        } else if (img == o.rep) {
            o.cnt += orb_popc(M);
        }
    }
    return o;
}

// The same with wk(k) returning p_k s (top step from the word).
template <class W>
XD_HD TorusOrbit torus_orbit(const TorusGeo &g, int ncos, W wk) {
    return torus_orbit_top(g, ncos, [&](int k, uint64_t *w, uint32_t *top) {
        *w = wk(k);
        return torus_top(g, *w, top);
    });
}

}  // namespace xd

// xd_sym.cu -- symmetry-adapted blocks of a site-permutation group.
//
// Basis (Sec. 3.10): the representative of an orbit is its smallest word;
// a representative r stays in the block of a 1-D representation chi when
// sum_{g in Stab(r)} chi(g) != 0.  The block is built on the device: every
// U(1) word is tested (a1 over the U(1) layout), the members are marked in a
// rank/select bitmap over U(1) ranks and compacted into the ascending
// representative list.
//
// Product (a4', derived from the projector of Sec. 3.10): with
// |r_chi> = (1/N_r) sum_g conj(chi(g)) g|r>, N_r = sqrt(|G| |Stab(r)|), the
// pull form of row r is
//     y_r = d(r) x_r + sum_{flips t} (J_b/2) chi(u_t) sqrt(|Stab(r'_t)|/|Stab(r)|) x_{r'_t}
// where r'_t = min_g g s_t is the representative of the flipped word s_t,
// u_t any element with u_t s_t = r'_t, and a target whose representative is
// not in the block contributes nothing.  The index of r'_t is its U(1) rank
// (two-table layout) followed by a rank/select lookup in the bitmap.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <unordered_map>

#include "xd_groups.h"
#include "xd_internal.cuh"
#include "xd_orbit.h"

namespace xd {

namespace {

constexpr int kThreads = 256;

// g s through byte tables: tab[g][c][v] is the image of the bits v << 8c.
__device__ __forceinline__ uint64_t act(const uint64_t *__restrict__ tab, int nchunk, int g,
                                        uint64_t s) {
    const uint64_t *t = tab + (size_t)g * nchunk * 256;
    uint64_t r = 0;
    for (int c = 0; c < nchunk; ++c) r |= __ldg(t + c * 256 + ((s >> (8 * c)) & 255));
    return r;
}

struct Orbit {
    uint64_t rep;  // smallest image
    int u;         // first g reaching it
    int cnt;       // number of g reaching it = |Stab(rep)|
};

__device__ __forceinline__ Orbit orbit_min_tables(const SymView &v, uint64_t s) {
    Orbit o{~0ull, 0, 0};
    for (int g = 0; g < v.G; ++g) {
        uint64_t t = act(v.act, v.nchunk, g, s);
        if (t < o.rep) {
            o.rep = t;
            o.u = g;
            o.cnt = 1;
        } else if (t == o.rep) {
            ++o.cnt;
        }
    }
    return o;
}

// Torus translations: (T_{a,b} s) puts in row y the row (y + b) mod Ly of s
// rotated by a (new bit x = old bit (x + a) mod Lx).  The smallest image must
// have the smallest possible top row, rot_a(row (Ly - 1 + b) mod Ly); only
// the (a, b) reaching that row are evaluated in full.
__device__ __forceinline__ uint64_t torus_image(uint64_t s, int a, int b, int Lx, int Ly,
                                                uint64_t rowmask) {
    uint64_t w = 0;
    for (int y = 0; y < Ly; ++y) {
        int ys = y + b;
        if (ys >= Ly) ys -= Ly;
        const uint64_t r = (s >> (Lx * ys)) & rowmask;
        const uint64_t rr = ((r >> a) | (r << (Lx - a))) & rowmask;
        w |= rr << (Lx * y);
    }
    return w;
}

// Smallest top row over the translations of s: rot-minimum of one of its rows.
__device__ __forceinline__ int torus_best(const SymView &v, uint64_t s) {
    const int Lx = v.tx, Ly = v.ty;
    const uint64_t rowmask = (1ull << Lx) - 1;
    int best = 1 << Lx;
    for (int y = 0; y < Ly; ++y) best = min(best, (int)__ldg(v.minrot + ((s >> (Lx * y)) & rowmask)));
    return best;
}

// Merges into o the translation images of s whose top row is `best` (its
// smallest top row); tg maps (a, b) to group indices.  Only the (a, b) that
// bring a row with rot-minimum `best` to the top, rotated to it, are formed.
__device__ __forceinline__ void torus_scan(const SymView &v, uint64_t s, int best, const int16_t *tg,
                                           Orbit &o) {
    const int Lx = v.tx, Ly = v.ty;
    const uint64_t rowmask = (1ull << Lx) - 1;
    for (int b = 0; b < Ly; ++b) {
        int yt = Ly - 1 + b;
        if (yt >= Ly) yt -= Ly;
        const uint32_t row = (uint32_t)((s >> (Lx * yt)) & rowmask);
        if (__ldg(v.minrot + row) != best) continue;
        uint32_t am = __ldg(v.amask + row);
        while (am) {
            const int a = __ffs(am) - 1;
            am &= am - 1;
            const uint64_t w = torus_image(s, a, b, Lx, Ly, rowmask);
            if (w < o.rep) {
                o.rep = w;
                o.u = __ldg(tg + a + Lx * b);
                o.cnt = 1;
            } else if (w == o.rep) {
                ++o.cnt;
            }
        }
    }
}

__device__ __forceinline__ Orbit orbit_min_torus(const SymView &v, uint64_t s) {
    Orbit o{~0ull, 0, 0};
    torus_scan(v, s, torus_best(v, s), v.tg, o);
    return o;
}

// Translations times point operations: G is the union of the cosets T p_k,
// so min_G = min over k of the translation minimum of p_k s.  Only the cosets
// whose smallest top row is the smallest of all are scanned in full.
// w(k) returns p_k s (p_0 = identity).
template <class W>
__device__ __forceinline__ Orbit coset_search(const SymView &v, W w) {
    int gb = torus_best(v, w(0));
    uint32_t sel = 1;  // cosets reaching gb (tnp <= 32 here)
    for (int k = 1; k < v.tnp; ++k) {
        const int bk = torus_best(v, w(k));
        if (bk < gb) {
            gb = bk;
            sel = 1u << k;
        } else if (bk == gb) {
            sel |= 1u << k;
        }
    }
    Orbit o{~0ull, 0, 0};
    const int T = v.tx * v.ty;
    while (sel) {
        const int k = __ffs(sel) - 1;
        sel &= sel - 1;
        torus_scan(v, w(k), gb, v.tg + k * T, o);
    }
    return o;
}

__device__ __forceinline__ Orbit orbit_min_cosets(const SymView &v, uint64_t s) {
    if (v.tnp <= 32)
        return coset_search(v, [&](int k) { return k ? act(v.act, v.nchunk, __ldg(v.tpp + k), s) : s; });
    Orbit o{~0ull, 0, 0};
    const int T = v.tx * v.ty;
    for (int k = 0; k < v.tnp; ++k) {
        const uint64_t w = k ? act(v.act, v.nchunk, __ldg(v.tpp + k), s) : s;
        torus_scan(v, w, torus_best(v, w), v.tg + k * T, o);
    }
    return o;
}

// Ring rotations T_n (i -> i + n mod N) and reflections R_n (i -> n - i mod
// N): T_n s = rotr(s, n) and R_n s = rotr(rev(s), N - 1 - n) on N-bit words.
// The smallest image has the longest run of zeros at its top, so only the
// rotations that bring a longest cyclic zero run of the word there are
// evaluated: z & rotr(z, 1) & ... & rotr(z, L - 1) marks the starts q of the
// runs of length >= L (z = zero bits of the word), and the run starting at q
// reaches the top under rotr(., (q + L) mod N).
__device__ __forceinline__ uint64_t ring_rotr(uint64_t w, int j, int N, uint64_t mask) {
    return j == 0 ? w : (((w >> j) | (w << (N - j))) & mask);
}

__device__ __forceinline__ Orbit orbit_min_ring(const SymView &v, uint64_t s) {
    const int N = v.cn;
    const uint64_t mask = N == 64 ? ~0ull : ((1ull << N) - 1);
    Orbit o{~0ull, 0, 0};
    for (int refl = 0; refl <= v.cdih; ++refl) {
        const uint64_t w = refl ? (__brevll(s) >> (64 - N)) : s;
        const uint64_t z = ~w & mask;
        if (z == 0) {  // all ones: every element fixes the word
            o.rep = w;
            o.u = __ldg(v.cg);
            o.cnt = v.G;
            return o;
        }
        uint64_t r = z;
        int L = 1;
        while (L < N) {
            const uint64_t r2 = r & ring_rotr(z, L, N, mask);
            if (!r2) break;
            r = r2;
            ++L;
        }
        while (r) {
            const int q = __ffsll((long long)r) - 1;
            r &= r - 1;
            int n = q + L;
            if (n >= N) n -= N;
            const uint64_t img = ring_rotr(w, n, N, mask);
            if (img <= o.rep) {
                int m = n;
                if (refl) {
                    m = N - 1 - n;
                    if (m < 0) m += N;
                }
                const int g = __ldg(v.cg + refl * N + m);
                if (img < o.rep) {
                    o.rep = img;
                    o.u = g;
                    o.cnt = 1;
                } else {
                    ++o.cnt;
                }
            }
        }
    }
    return o;
}

// Narrowing search of xd_orbit.h (tori with at most 8 rows); rowtab in
// global or shared memory.
__device__ __forceinline__ TorusGeo torus_view(const SymView &v, const uint16_t *rowtab, const uint16_t *cut) {
    TorusGeo g;
    g.Lx = v.tx;
    g.Ly = v.ty;
    g.N = v.N;
    g.rowmask = (1u << v.tx) - 1;
    g.nmask = ~0ull >> (64 - v.N);
    g.rep1 = v.trep1;
    g.rowtab = rowtab;
    g.cut = cut;
    return g;
}

__device__ __forceinline__ Orbit torus_result(const SymView &v, const TorusOrbit &t) {
    Orbit o;
    o.rep = t.rep;
    o.cnt = t.cnt;
    o.u = __ldg(v.tg + t.k * v.N + (t.q & 7) + v.tx * (t.q >> 3));
    return o;
}

__device__ __forceinline__ Orbit orbit_min_narrow(const SymView &v, const TorusGeo &g, uint64_t s) {
    return torus_result(v, torus_orbit(g, v.tnp ? v.tnp : 1, [&](int k) {
                            return k ? act(v.act, v.nchunk, __ldg(v.tpp + k), s) : s;
                        }));
}

__device__ __forceinline__ Orbit orbit_min(const SymView &v, uint64_t s) {
    if (v.tx) {
        if (v.ty <= 8) return orbit_min_narrow(v, torus_view(v, v.rowtab, v.cut), s);
        return v.tnp ? orbit_min_cosets(v, s) : orbit_min_torus(v, s);
    }
    return v.cn ? orbit_min_ring(v, s) : orbit_min_tables(v, s);
}

__device__ __forceinline__ uint64_t find_block(const int64_t *__restrict__ hi_off, uint64_t lo,
                                               uint64_t hi, int64_t r) {
    while (lo < hi) {
        uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(hi_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t u1_state(const U1View &u, int64_t k, uint64_t &h) {
    // h: a lower bound hint for the block (updated)
    while (__ldg(u.hi_off + h + 1) <= k) ++h;
    int m = u.nup - __popcll(h);
    uint32_t l = __ldg(u.lo_list + __ldg(u.lo_off + m) + (uint32_t)(k - __ldg(u.hi_off + h)));
    return (h << u.L) | l;
}

// Membership test of the 64 U(1) states of word w.
__device__ uint64_t member_word(const SymView &v, const double *__restrict__ chi, int64_t w,
                                int *nmem) {
    const U1View &u = v.u1;
    int64_t k0 = w * 64, k1 = min(k0 + 64, u.dim);
    uint64_t h = find_block(u.hi_off, 0, (1ull << u.P) - 1, k0);
    uint64_t bits = 0;
    for (int64_t k = k0; k < k1; ++k) {
        uint64_t s = u1_state(u, k, h);
        double cr = 0.0, ci = 0.0;
        bool is_rep = true;
        if (v.tx || v.cn) {
            // a fast orbit search decides; the character sum runs on representatives only
            is_rep = orbit_min(v, s).rep == s;
            for (int g = 0; g < v.G && is_rep; ++g)
                if (act(v.act, v.nchunk, g, s) == s) {
                    cr += chi[2 * g];
                    ci += chi[2 * g + 1];
                }
        } else {
            for (int g = 0; g < v.G && is_rep; ++g) {
                uint64_t t = act(v.act, v.nchunk, g, s);
                if (t < s) is_rep = false;
                if (t == s) {
                    cr += chi[2 * g];
                    ci += chi[2 * g + 1];
                }
            }
        }
        if (is_rep && cr * cr + ci * ci > 0.25) bits |= 1ull << (k - k0);
    }
    *nmem = __popcll(bits);
    return bits;
}

__global__ void k_mark(SymView v, const double *__restrict__ chi, int64_t nwords,
                       uint64_t *__restrict__ bits, int64_t *__restrict__ cnt) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x) {
        int n;
        bits[w] = member_word(v, chi, w, &n);
        cnt[w] = n;
    }
}

__global__ void k_compact(SymView v, int64_t nwords, const uint64_t *__restrict__ bits,
                          const int64_t *__restrict__ cum, uint64_t *__restrict__ reps,
                          uint16_t *__restrict__ stab) {
    const U1View &u = v.u1;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x) {
        uint64_t b = bits[w];
        if (!b) continue;
        int64_t k0 = w * 64;
        uint64_t h = find_block(u.hi_off, 0, (1ull << u.P) - 1, k0);
        int64_t out = cum[w];
        while (b) {
            int j = __ffsll((long long)b) - 1;
            b &= b - 1;
            uint64_t s = u1_state(u, k0 + j, h);
            reps[out] = s;
            stab[out] = (uint16_t)orbit_min(v, s).cnt;
            ++out;
        }
    }
}

// rank/select words: member bits and the number of members before the word
__global__ void k_interleave(int64_t nwords, const uint64_t *__restrict__ bits,
                             const int64_t *__restrict__ cum, ulonglong2 *__restrict__ rs) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (int64_t)gridDim.x * blockDim.x)
        rs[w] = make_ulonglong2(bits[w], (unsigned long long)cum[w]);
}

// ---- exclusive scan of int64 counts (three phases, fixed order)
constexpr int kScanChunk = 4096;

__global__ void k_scan_sums(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t red[kThreads];
    int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int64_t s = 0;
    for (int64_t i = base + threadIdx.x; i < min(base + kScanChunk, n); i += blockDim.x) s += in[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

__global__ void k_scan_serial(int64_t *__restrict__ sums, int64_t n) {
    if (threadIdx.x || blockIdx.x) return;
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t t = sums[i];
        sums[i] = run;
        run += t;
    }
    sums[n] = run;
}

__global__ void k_scan_apply(const int64_t *__restrict__ in, int64_t n,
                             const int64_t *__restrict__ sums, int64_t *__restrict__ out) {
    // one thread walks a sub-chunk; the block scans the sub-chunk totals
    __shared__ int64_t part[kThreads + 1];
    const int per = kScanChunk / kThreads;
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * per;
    int64_t s = 0;
    for (int k = 0; k < per; ++k)
        if (base + k < n) s += in[base + k];
    part[threadIdx.x + 1] = s;
    if (threadIdx.x == 0) part[0] = 0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 1; t <= kThreads; ++t) part[t] += part[t - 1];
    __syncthreads();
    int64_t run = sums[blockIdx.x] + part[threadIdx.x];
    for (int k = 0; k < per; ++k)
        if (base + k < n) {
            out[base + k] = run;
            run += in[base + k];
        }
}

template <bool CPLX>
struct Val;
template <>
struct Val<false> {
    using T = double;
};
template <>
struct Val<true> {
    using T = double2;
};

// Row r of y = H x (see the file header).  sq[a] = sqrt(a), sq[G + 1 + m] =
// 1 / sqrt(m), so sqrt(|Stab(r')| / |Stab(r)|) = sq[|Stab(r')|] sq[G + 1 + |Stab(r)|].
// COS: translations times at most kMaxCos point operations; the point images
// p_k s of the row are formed once and those of a flipped word by one XOR
// with the point images of the bond masks (kept in shared memory).
constexpr int kMaxCos = 12;

// Bonds of the product sorted by coupling, in chunks of 64 (bit q of chunk c
// is sorted bond 64 c + q); a group is a run of equal coupling inside one
// chunk (the layout of xd_ham_s::d_symgrp).
struct SymBonds {
    const uint64_t *smask;  // [nb] site masks, sorted order
    const uint64_t *gmask;  // [ngrp] bits of the group in its chunk
    const double *ghalf;    // [ngrp] J/2
    const uint16_t *perm;   // [nb] bond id of each sorted bond
    const uint16_t *goff;   // [nchunk + 1] first group of each chunk
    int ngrp, nchunk;
};

__host__ __device__ inline size_t symgrp_words(int nb, int ngrp) {
    const int nchunk = (nb + 63) / 64;
    return (size_t)nb + 2 * (size_t)ngrp + ((size_t)nb + nchunk + 1 + 3) / 4;
}

__host__ __device__ inline SymBonds symgrp_view(const uint64_t *base, int nb, int ngrp) {
    SymBonds v;
    v.smask = base;
    v.gmask = base + nb;
    v.ghalf = (const double *)(base + nb + ngrp);
    v.perm = (const uint16_t *)(base + nb + 2 * ngrp);
    v.goff = v.perm + nb;
    v.ngrp = ngrp;
    v.nchunk = (nb + 63) / 64;
    return v;
}

template <bool CPLX, bool COS>
__global__ void __launch_bounds__(kThreads) k_sym_apply(SymView v, SymBonds sbo, int nb, double jq,
                                                        const double *__restrict__ chi,
                                                        const double *__restrict__ sq,
                                                        const typename Val<CPLX>::T *__restrict__ x,
                                                        typename Val<CPLX>::T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ngrp = sbo.ngrp, nchunk = sbo.nchunk;
    uint64_t *sm_smask = (uint64_t *)smem;                   // [nb] sorted bonds
    uint64_t *sm_gmask = sm_smask + nb;                      // [ngrp]
    double *sm_ghalf = (double *)(sm_gmask + ngrp);          // [ngrp]
    double *sm_chi = sm_ghalf + ngrp;                        // [G][2]
    double *sm_sq = sm_chi + 2 * v.G;                        // [2 (G+1)]
    uint64_t *sm_pm = (uint64_t *)(sm_sq + 2 * (v.G + 1));  // COS: [tnp - 1][nb]
    uint64_t *sm_ps = sm_pm + (COS ? (v.tnp - 1) * nb : 0);   // COS: [tnp - 1][threads]
    uint64_t *sm_st = sm_ps + (COS ? (v.tnp - 1) * kThreads : 0);  // COS: [tnp - 1][threads] row states
    uint16_t *sm_rowtab = (uint16_t *)(sm_st + (COS ? 2 * (v.tnp - 1) * kThreads : 0));  // [256]
    uint16_t *sm_cut = sm_rowtab + 256;                            // [2^(2 tx)] when v.cut
    uint16_t *sm_krow = sm_cut + (v.cut ? (1 << (2 * v.tx)) : 0);  // [max(1, tnp)][nb]
    uint16_t *sm_perm = sm_krow + max(1, v.tnp) * nb;              // [nb]
    uint16_t *sm_goff = sm_perm + nb;                              // [nchunk + 1]
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        sm_smask[q] = sbo.smask[q];
        sm_perm[q] = sbo.perm[q];
    }
    for (int q = threadIdx.x; q < ngrp; q += blockDim.x) {
        sm_gmask[q] = sbo.gmask[q];
        sm_ghalf[q] = sbo.ghalf[q];
    }
    for (int q = threadIdx.x; q <= nchunk; q += blockDim.x) sm_goff[q] = sbo.goff[q];
    for (int g = threadIdx.x; g < 2 * v.G; g += blockDim.x) sm_chi[g] = chi[g];
    for (int q = threadIdx.x; q < 2 * (v.G + 1); q += blockDim.x) sm_sq[q] = sq[q];
    if constexpr (COS)
        for (int q = threadIdx.x; q < (v.tnp - 1) * nb; q += blockDim.x) sm_pm[q] = v.pm[q];
    const bool narrow = v.tx && v.ty <= 8;
    if (narrow) {
        for (int q = threadIdx.x; q < (1 << v.tx); q += blockDim.x) sm_rowtab[q] = v.rowtab[q];
        if (v.cut)
            for (int q = threadIdx.x; q < (1 << (2 * v.tx)); q += blockDim.x) sm_cut[q] = v.cut[q];
        for (int q = threadIdx.x; q < max(1, v.tnp) * nb; q += blockDim.x) sm_krow[q] = v.krow[q];
    }
    // incremental top step (row states, rows of at most 7 sites): translations
    // alone, or the coset form
    const bool rows = narrow && v.tx <= 7 && (COS || v.tnp == 0);
    const TorusGeo tgeo = torus_view(v, sm_rowtab, v.cut ? sm_cut : nullptr);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < v.dim;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = __ldg(v.reps + r);
        // translations alone, real blocks: the three smallest rows of s; otherwise
        // the row state of s (the complex form keeps its registers below 64 so)
        constexpr bool kTop3 = !COS && !CPLX;
        uint64_t PM = 0, PA = 0;
        RowTop3 t3;
        if (rows && kTop3) torus_top3(tgeo, s, t3);
        else if (rows) torus_rows(tgeo, s, PM, PA);
        if constexpr (COS) {
            for (int k = 1; k < v.tnp; ++k) {
                const uint64_t w = act(v.act, v.nchunk, __ldg(v.tpp + k), s);
                sm_ps[(k - 1) * kThreads + threadIdx.x] = w;
                if (rows) {
                    uint64_t pm, pa;
                    torus_rows(tgeo, w, pm, pa);
                    sm_st[2 * ((k - 1) * kThreads + threadIdx.x)] = pm;
                    sm_st[2 * ((k - 1) * kThreads + threadIdx.x) + 1] = pa;
                }
            }
        }
        // sum over flips of sqrt(|Stab(r')|) chi(u) x_{r'}, per group of equal
        // coupling, times J/2; 1/sqrt(|Stab(r)|) once at the end
        double ar = 0.0, ai = 0.0, dsub = 0.0;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int b0 = 64 * ch, nq = min(64, nb - b0);
            // flipping bonds of the chunk (antiparallel sites) as the set bits
            // of F, so that a warp takes as many steps as its rows have flips
            uint64_t F = 0;
            for (int q = 0; q < nq; ++q) {
                const uint64_t mq = sm_smask[b0 + q];
                const uint64_t t = s & mq;
                F |= (uint64_t)(t != 0 && t != mq) << q;
            }
            for (int g = sm_goff[ch]; g < sm_goff[ch + 1]; ++g) {
                uint64_t Fg = F & sm_gmask[g];
                const double hb = sm_ghalf[g];
                dsub += hb * __popcll(Fg);
                double gr = 0.0, gi = 0.0;
                while (Fg) {
                    const int bs = b0 + __ffsll((long long)Fg) - 1;
                    Fg &= Fg - 1;
                    const uint64_t mk = sm_smask[bs];
                    const int b = sm_perm[bs];  // bond id (point-image and row tables)
                    Orbit o;
                    if (rows) {
                        // p_k of the flipped word and its top step: from the three smallest
                        // rows of s (kTop3), or from the row state of p_k s refreshed in the
                        // two rows of the flip
                        o = torus_result(v, torus_orbit_top(tgeo, COS ? v.tnp : 1,
                                                            [&](int k, uint64_t *w, uint32_t *top) {
                            if (kTop3) {
                                *w = s ^ mk;
                                const uint32_t rr = sm_krow[b];
                                return torus_top_flip(tgeo, t3, *w, rr & 0xffu, rr >> 8, top);
                            }
                            uint64_t pm = PM, pa = PA;
                            if (COS && k) {
                                const int e = (k - 1) * kThreads + threadIdx.x;
                                *w = sm_ps[e] ^ sm_pm[(k - 1) * nb + b];
                                pm = sm_st[2 * e];
                                pa = sm_st[2 * e + 1];
                            } else {
                                *w = s ^ mk;
                            }
                            const uint32_t rr = sm_krow[k * nb + b];
                            torus_rows_set(tgeo, pm, pa, *w, rr & 0xffu);
                            torus_rows_set(tgeo, pm, pa, *w, rr >> 8);
                            return torus_top_rows(tgeo, pm, pa, top);
                        }));
                    } else if constexpr (COS) {
                        o = coset_search(v, [&](int k) {
                            return k ? sm_ps[(k - 1) * kThreads + threadIdx.x] ^ sm_pm[(k - 1) * nb + b] : s ^ mk;
                        });
                    } else {
                        o = narrow ? orbit_min_narrow(v, tgeo, s ^ mk) : orbit_min(v, s ^ mk);
                    }
                    const int64_t k = __ldg(v.u1.hi_off + (o.rep >> v.u1.L)) +
                                      (int64_t)__ldg(v.u1.lo_rank + (o.rep & v.u1.lomask));
                    const ulonglong2 wc = __ldg(v.rs + (k >> 6));
                    const uint64_t word = wc.x;
                    if (!((word >> (k & 63)) & 1)) continue;
                    const int64_t c = (int64_t)wc.y + __popcll(word & ((1ull << (k & 63)) - 1));
                    const double a = sm_sq[o.cnt];
                    if constexpr (CPLX) {
                        const double2 xc = x[c];
                        const double tr = a * xc.x, ti = a * xc.y;
                        const double chr = sm_chi[2 * o.u], chim = sm_chi[2 * o.u + 1];
                        gr += chr * tr - chim * ti;
                        gi += chr * ti + chim * tr;
                    } else {
                        gr = fma(a * sm_chi[2 * o.u], x[c], gr);
                    }
                }
                ar = fma(hb, gr, ar);
                ai = fma(hb, gi, ai);
            }
        }
        const double d = jq - dsub;
        const double isr = sm_sq[v.G + 1 + __ldg(v.stab + r)];
        if constexpr (CPLX) {
            const double2 xr = x[r];
            y[r] = make_double2(d * xr.x + isr * ar, d * xr.y + isr * ai);
        } else {
            y[r] = d * x[r] + isr * ar;
        }
    }
}

// Per-bond contributions C(b) = Re sum_r conj(g_r) [bond-b part of row r],
// reduced per CTA into part[cta][b] (fixed order).
constexpr int kChunk = 128;

template <bool CPLX, bool ZZ = false>
__global__ void __launch_bounds__(kThreads) k_sym_bilinear(SymView v, const uint64_t *__restrict__ masks,
                                                           int nb, int b0, const double *__restrict__ chi,
                                                           const double *__restrict__ sq,
                                                           const typename Val<CPLX>::T *__restrict__ g,
                                                           const typename Val<CPLX>::T *__restrict__ x,
                                                           double *__restrict__ part) {
    __shared__ double acc[kThreads / 32][kChunk];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nbc = min(kChunk, nb - b0);
    for (int b = lane; b < nbc; b += 32) acc[warp][b] = 0.0;
    __syncwarp();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t rounds = (v.dim + stride - 1) / stride;
    for (int64_t it = 0; it < rounds; ++it) {
        const int64_t r = it * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool valid = r < v.dim;
        uint64_t s = 0;
        int mr = 1;
        double gr = 0, gi = 0, xr = 0, xi = 0;
        if (valid) {
            s = v.reps[r];
            mr = v.stab[r];
            if constexpr (CPLX) {
                gr = g[r].x; gi = g[r].y; xr = x[r].x; xi = x[r].y;
            } else {
                gr = g[r]; xr = x[r];
            }
        }
        for (int b = 0; b < nbc; ++b) {
            double val = 0.0;
            if (valid) {
                const uint64_t mk = masks[b0 + b];
                const uint64_t t = s & mk;
                // Re conj(g_r) * (term) ; diagonal term is +-1/4 x_r
                const double diag = (t == 0 || t == mk) ? 0.25 : -0.25;
                val = diag * (gr * xr + gi * xi);
                if (!ZZ && !(t == 0 || t == mk)) {
                    const Orbit o = orbit_min(v, s ^ mk);
                    const int64_t k = __ldg(v.u1.hi_off + (o.rep >> v.u1.L)) +
                                      (int64_t)__ldg(v.u1.lo_rank + (o.rep & v.u1.lomask));
                    const ulonglong2 wc = __ldg(v.rs + (k >> 6));
                    const uint64_t word = wc.x;
                    if ((word >> (k & 63)) & 1) {
                        const int64_t c = (int64_t)wc.y +
                                          __popcll(word & ((1ull << (k & 63)) - 1));
                        const double a = 0.5 * sq[o.cnt] * sq[v.G + 1 + mr];
                        const double cr = a * chi[2 * o.u], ci = a * chi[2 * o.u + 1];
                        double tr, ti;
                        if constexpr (CPLX) {
                            tr = cr * x[c].x - ci * x[c].y;
                            ti = cr * x[c].y + ci * x[c].x;
                        } else {
                            tr = cr * x[c];
                            ti = ci * x[c];
                        }
                        val += gr * tr + gi * ti;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
            if (lane == 0) acc[warp][b] += val;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbc; b += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += acc[w][b];
        part[(size_t)blockIdx.x * nb + b0 + b] = s;
    }
}

// dJ[b] = mean over the bond orbit of sum_c part[c][b']
__global__ void k_orbit_mean(const double *__restrict__ part, int rows, int nb,
                             const int32_t *__restrict__ orbit, double *__restrict__ out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double s = 0.0;
    int n = 0;
    for (int q = 0; q < nb; ++q) {
        if (orbit[q] != orbit[b]) continue;
        ++n;
        for (int c = 0; c < rows; ++c) s += part[(size_t)c * nb + q];
    }
    out[b] = s / n;
}

}  // namespace

template <typename E>
static xd_status upload(E **dst, const std::vector<E> &v) {
    XD_CUDA(dev_malloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(E)));
    XD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
    return XD_OK;
}

static xd_status make_tables(xd_basis_s *b) {
    const int N = b->N, G = b->G;
    GroupTables T;
    group_tables(N, G, b->perms.data(), (const int32_t *)b->bonds.data(), b->nb, &T);
    b->nchunk = T.nchunk;
    if (T.tx) {
        XD_TRY(upload(&b->d_minrot, T.minrot));
        XD_TRY(upload(&b->d_amask, T.amask));
        std::vector<uint16_t> rowtab(T.minrot.size());
        for (size_t r = 0; r < rowtab.size(); ++r) rowtab[r] = (uint16_t)(T.minrot[r] | (T.amask[r] << 8));
        XD_TRY(upload(&b->d_rowtab, rowtab));
        if (!T.cut.empty()) XD_TRY(upload(&b->d_cut, T.cut));
        const int ncos = std::max(1, T.tnp), nb = b->nb;
        std::vector<uint16_t> krow((size_t)ncos * nb);
        for (int k = 0; k < ncos; ++k)
            for (int q = 0; q < nb; ++q) {
                const uint64_t m = k ? T.pm[(size_t)(k - 1) * nb + q]
                                     : (1ull << b->bonds[q].i) | (1ull << b->bonds[q].j);
                const int lo = __builtin_ctzll(m) / T.tx, hi = (63 - __builtin_clzll(m)) / T.tx;
                krow[(size_t)k * nb + q] = (uint16_t)(lo | (hi << 8));
            }
        XD_TRY(upload(&b->d_krow, krow));
        b->trep1 = torus_geo(T.tx, T.ty, nullptr).rep1;
        XD_TRY(upload(&b->d_tg, T.tg));
        XD_TRY(upload(&b->d_tpp, T.tpp));
        if (T.tnp) XD_TRY(upload(&b->d_pm, T.pm));
        b->tx = T.tx;
        b->ty = T.ty;
        b->tnp = T.tnp;
    } else if (T.cn) {
        XD_TRY(upload(&b->d_cg, T.cg));
        b->cn = T.cn;
        b->cdih = T.cdih;
    }
    XD_TRY(upload(&b->d_act, T.act));
    std::vector<double> chi(2 * G);
    for (int g = 0; g < G; ++g) {
        chi[2 * g] = b->chi_re[g];
        chi[2 * g + 1] = b->chi_im[g];
    }
    XD_TRY(upload(&b->d_chi, chi));
    return XD_OK;
}

xd_status sym_build(xd_basis_s *b) {
    XD_TRY(make_tables(b));
    const int64_t nwords = (b->dim_u1 + 63) / 64;
    const int64_t nchunks = (nwords + kScanChunk - 1) / kScanChunk;
    const int grid = grid_for(nwords, kThreads, 16);
    // temporaries of the build, released on every path (the scan's as soon
    // as the count is known, to keep the peak down)
    uint64_t *d_bits = nullptr;
    int64_t *d_cum = nullptr, *cnt = nullptr, *sums = nullptr;
    const char *what = "cudaMalloc(symmetric basis build)";
    cudaError_t e = dev_malloc((void **)&d_bits, std::max<int64_t>(1, nwords) * sizeof(uint64_t));
    if (e == cudaSuccess) e = dev_malloc((void **)&d_cum, (nwords + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = dev_malloc((void **)&cnt, std::max<int64_t>(1, nwords) * sizeof(int64_t));
    if (e == cudaSuccess) e = dev_malloc((void **)&sums, (nchunks + 1) * sizeof(int64_t));
    int64_t total = 0;
    if (e == cudaSuccess) {
        what = "symmetric basis build";
        const SymView v = b->symview();
        k_mark<<<grid, kThreads>>>(v, b->d_chi, nwords, d_bits, cnt);
        k_scan_sums<<<(unsigned)std::max<int64_t>(1, nchunks), kThreads>>>(cnt, nwords, sums);
        k_scan_serial<<<1, 1>>>(sums, nchunks);
        k_scan_apply<<<(unsigned)std::max<int64_t>(1, nchunks), kThreads>>>(cnt, nwords, sums, d_cum);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(&total, sums + nchunks, sizeof total, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(d_cum + nwords, &total, sizeof total, cudaMemcpyHostToDevice);
    }
    cudaFree(cnt);
    cudaFree(sums);
    if (e == cudaSuccess) {
        b->dim = total;
        what = "symmetric basis compaction";
        e = dev_malloc((void **)&b->d_reps, std::max<int64_t>(1, total) * sizeof(uint64_t));
        if (e == cudaSuccess) e = dev_malloc((void **)&b->d_stab, std::max<int64_t>(1, total) * sizeof(uint16_t));
        if (e == cudaSuccess) {
            const SymView v = b->symview();
            k_compact<<<grid, kThreads>>>(v, nwords, d_bits, d_cum, b->d_reps, b->d_stab);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = dev_malloc((void **)&b->d_rs, std::max<int64_t>(1, nwords) * sizeof(ulonglong2));
        if (e == cudaSuccess) {
            k_interleave<<<grid, kThreads>>>(nwords, d_bits, d_cum, b->d_rs);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(d_bits);
    cudaFree(d_cum);
    if (e != cudaSuccess) return cuda_status(e, what);
    return XD_OK;
}

// Per-Hamiltonian tables: sqrt(a) and 1/sqrt(a) for a in [1, G] and the
// orbit id of every bond under the group (bilinear forms are averaged over
// bond orbits).
xd_status sym_ham_tables(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const int G = b->G, nb = b->nb;
    const size_t nsq = 2 * (size_t)(G + 1);
    std::vector<double> tab(nsq + (nb + 1) / 2 + 1, 0.0);
    for (int a = 1; a <= G; ++a) {
        tab[a] = sqrt((double)a);
        tab[G + 1 + a] = 1.0 / sqrt((double)a);
    }
    std::vector<int32_t> orb(nb, -1);
    bond_orbits(b->N, G, b->perms.data(), (const int32_t *)b->bonds.data(), nb, orb.data());
    memcpy(tab.data() + nsq, orb.data(), nb * sizeof(int32_t));
    XD_CUDA(dev_malloc((void **)&h->d_symtab, tab.size() * sizeof(double)));
    XD_CUDA(cudaMemcpy(h->d_symtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
    return XD_OK;
}

xd_status sym_bond_groups(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const int nb = b->nb, nchunk = (nb + 63) / 64;
    if (nb > 65535) {
        set_error("symmetric product: %d bonds (at most 65535)", nb);
        return XD_ERANGE;
    }
    std::vector<int> order(nb);
    for (int q = 0; q < nb; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return h->J[p] < h->J[q]; });
    std::vector<uint64_t> gmask;
    std::vector<double> ghalf;
    std::vector<uint16_t> goff(nchunk + 1, 0);
    for (int c = 0; c < nchunk; ++c) {
        goff[c] = (uint16_t)gmask.size();
        for (int q = 64 * c; q < std::min(nb, 64 * c + 64); ++q) {
            const double J = h->J[order[q]];
            if (q == 64 * c || J != h->J[order[q - 1]]) {
                gmask.push_back(0);
                ghalf.push_back(0.5 * J);
            }
            gmask.back() |= 1ull << (q - 64 * c);
        }
    }
    goff[nchunk] = (uint16_t)gmask.size();
    const int ngrp = (int)gmask.size();
    std::vector<uint64_t> tab(symgrp_words(nb, ngrp), 0);
    for (int q = 0; q < nb; ++q)
        tab[q] = (1ull << b->bonds[order[q]].i) | (1ull << b->bonds[order[q]].j);
    for (int g = 0; g < ngrp; ++g) {
        tab[nb + g] = gmask[g];
        memcpy(&tab[nb + ngrp + g], &ghalf[g], sizeof(double));
    }
    uint16_t *u16 = (uint16_t *)(tab.data() + nb + 2 * ngrp);
    for (int q = 0; q < nb; ++q) u16[q] = (uint16_t)order[q];
    for (int c = 0; c <= nchunk; ++c) u16[nb + c] = goff[c];
    if (h->d_symgrp && h->sym_ngrp != ngrp) {
        cudaFree(h->d_symgrp);
        h->d_symgrp = nullptr;
    }
    if (!h->d_symgrp) XD_CUDA(dev_malloc((void **)&h->d_symgrp, tab.size() * sizeof(uint64_t)));
    XD_CUDA(cudaMemcpy(h->d_symgrp, tab.data(), tab.size() * sizeof(uint64_t), cudaMemcpyHostToDevice));
    h->sym_ngrp = ngrp;
    return XD_OK;
}

struct SymWork {
    const double *sq;
    const int32_t *orbit;
    double *part;
};

static xd_status sym_work(const xd_ham_s *h, int grid, SymWork *w) {
    const xd_basis_s *b = h->b;
    const size_t nsq = 2 * (size_t)(b->G + 1);
    w->sq = h->d_symtab;
    w->orbit = (const int32_t *)(h->d_symtab + nsq);
    w->part = nullptr;
    if (grid > 0) {
        XD_TRY(ensure_partials(const_cast<xd_ham_s *>(h), (size_t)grid * b->nb * sizeof(double)));
        w->part = h->d_part;
    }
    return XD_OK;
}

xd_status sym_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const int nb = b->nb, G = b->G;
    SymWork w;
    XD_TRY(sym_work(h, 0, &w));
    const SymView v = b->symview();
    const SymBonds sbo = symgrp_view(h->d_symgrp, nb, h->sym_ngrp);
    double jq = 0.0;
    for (int q = 0; q < nb; ++q) jq += h->J[q];
    jq *= 0.25;
    // u16 tables: rows of the narrowing search, the bonds' rows, bond ids, first groups
    const size_t tabs = (256 + (b->d_cut ? ((size_t)1 << (2 * b->tx)) : 0) + (size_t)std::max(1, b->tnp) * nb + nb +
                         sbo.nchunk + 1) * sizeof(uint16_t);
    size_t smem = (size_t)nb * 8 + (size_t)sbo.ngrp * 16 + 2 * G * sizeof(double) +
                  2 * (size_t)(G + 1) * sizeof(double) + tabs;
    // coset form: point images of the bond masks, per-thread images of the row and their row states
    const size_t smem_cos = smem + (size_t)std::max(0, b->tnp - 1) * (nb + 3 * kThreads) * sizeof(uint64_t);
    int optin = 0;
    {
        int dev = 0;
        XD_CUDA(cudaGetDevice(&dev));
        XD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (smem > (size_t)optin) {
            set_error("symmetric product: %d bonds and %d group elements need %zu bytes of shared memory",
                      nb, G, smem);
            return XD_ERANGE;
        }
    }
    int grid = grid_for(v.dim, kThreads, 8);
    // coset form when the point images of the bond masks fit beside the rest
    const bool cos = v.tx && v.tnp > 1 && v.tnp <= kMaxCos && smem_cos <= (size_t)optin;
    if (cos) smem = smem_cos;
    if (dt == XD_C128) {
        auto kern = cos ? k_sym_apply<true, true> : k_sym_apply<true, false>;
        XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kThreads, smem, st>>>(v, sbo, nb, jq, b->d_chi, w.sq, (const double2 *)x, (double2 *)y);
    } else {
        auto kern = cos ? k_sym_apply<false, true> : k_sym_apply<false, false>;
        XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, kThreads, smem, st>>>(v, sbo, nb, jq, b->d_chi, w.sq, (const double *)x, (double *)y);
    }
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status sym_bilinear(const xd_ham_s *h, const void *g, const void *x, xd_dtype dt, double *dJ,
                       cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const int nb = b->nb;
    const SymView v = b->symview();
    const int grid = grid_for(v.dim, kThreads, 4);
    SymWork w;
    XD_TRY(sym_work(h, grid, &w));
    const uint64_t *masks = (const uint64_t *)(h->d_bond + nb);
    for (int b0 = 0; b0 < nb; b0 += kChunk) {
        if (dt == XD_C128)
            k_sym_bilinear<true><<<grid, kThreads, 0, st>>>(v, masks, nb, b0, b->d_chi, w.sq,
                                                            (const double2 *)g, (const double2 *)x,
                                                            w.part);
        else
            k_sym_bilinear<false><<<grid, kThreads, 0, st>>>(v, masks, nb, b0, b->d_chi, w.sq,
                                                             (const double *)g, (const double *)x,
                                                             w.part);
        XD_CUDA(cudaGetLastError());
    }
    k_orbit_mean<<<(nb + 127) / 128, 128, 0, st>>>(w.part, grid, nb, w.orbit, dJ);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// Two-point correlations on a symmetry-adapted block: the pairs' orbits under
// the group become a list of site pairs (each unordered pair once) with an
// orbit id; the symmetric bond form of every listed pair (its diagonal part
// alone for Sz Sz) is averaged over its orbit, which is <psi| O_ij |psi> of
// the lifted state for every pair of the orbit (within a one-dimensional
// irrep the expectation value is constant on a pair orbit, Sec. 3.10).
xd_status sym_correlations(const xd_basis_s *b, const void *psi, xd_dtype dt, const int32_t *pairs, int npairs,
                           int kind, double *out) {
    const int N = b->N, G = b->G;
    std::vector<uint64_t> masks;
    std::vector<int32_t> orb;
    std::map<std::pair<int, int>, int> where;
    std::vector<int> slot(npairs);
    int norb = 0;
    for (int q = 0; q < npairs; ++q) {
        const int i = std::min(pairs[2 * q], pairs[2 * q + 1]), j = std::max(pairs[2 * q], pairs[2 * q + 1]);
        auto it = where.find({i, j});
        if (it == where.end()) {
            for (int g = 0; g < G; ++g) {
                const int32_t *pg = b->perms.data() + (size_t)g * N;
                const std::pair<int, int> e(std::min(pg[i], pg[j]), std::max(pg[i], pg[j]));
                if (where.count(e)) continue;
                where[e] = (int)masks.size();
                masks.push_back((1ull << e.first) | (1ull << e.second));
                orb.push_back(norb);
            }
            ++norb;
            it = where.find({i, j});
        }
        slot[q] = it->second;
    }
    const int nm = (int)masks.size();
    const SymView v = b->symview();
    const int grid = grid_for(v.dim, kThreads, 4);
    std::vector<double> sq(2 * (size_t)(G + 1), 0.0);
    for (int a = 1; a <= G; ++a) {
        sq[a] = sqrt((double)a);
        sq[G + 1 + a] = 1.0 / sqrt((double)a);
    }
    uint64_t *d_m = nullptr;
    int32_t *d_o = nullptr;
    double *d_sq = nullptr, *d_part = nullptr, *d_out = nullptr;
    cudaError_t e = dev_malloc((void **)&d_m, sizeof(uint64_t) * nm);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_o, sizeof(int32_t) * nm);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_sq, sizeof(double) * sq.size());
    if (e == cudaSuccess) e = dev_malloc((void **)&d_part, sizeof(double) * (size_t)grid * nm);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_out, sizeof(double) * nm);
    if (e == cudaSuccess) e = cudaMemcpy(d_m, masks.data(), sizeof(uint64_t) * nm, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_o, orb.data(), sizeof(int32_t) * nm, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_sq, sq.data(), sizeof(double) * sq.size(), cudaMemcpyHostToDevice);
    for (int b0 = 0; e == cudaSuccess && b0 < nm; b0 += kChunk) {
        if (dt == XD_C128) {
            if (kind) k_sym_bilinear<true, false><<<grid, kThreads>>>(v, d_m, nm, b0, b->d_chi, d_sq, (const double2 *)psi, (const double2 *)psi, d_part);
            else k_sym_bilinear<true, true><<<grid, kThreads>>>(v, d_m, nm, b0, b->d_chi, d_sq, (const double2 *)psi, (const double2 *)psi, d_part);
        } else {
            if (kind) k_sym_bilinear<false, false><<<grid, kThreads>>>(v, d_m, nm, b0, b->d_chi, d_sq, (const double *)psi, (const double *)psi, d_part);
            else k_sym_bilinear<false, true><<<grid, kThreads>>>(v, d_m, nm, b0, b->d_chi, d_sq, (const double *)psi, (const double *)psi, d_part);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_orbit_mean<<<(nm + 127) / 128, 128>>>(d_part, grid, nm, d_o, d_out);
        e = cudaGetLastError();
    }
    std::vector<double> val(nm, 0.0);
    if (e == cudaSuccess) e = cudaMemcpy(val.data(), d_out, sizeof(double) * nm, cudaMemcpyDeviceToHost);
    cudaFree(d_m);
    cudaFree(d_o);
    cudaFree(d_sq);
    cudaFree(d_part);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_status(e, "xd_correlations (symmetric block)");
    // a pair i = j has a one-bit mask that never flips: <psi|psi>/4 = (Sz_i)^2;
    // S_i.S_i = 3/4 <psi|psi> is three times that
    for (int q = 0; q < npairs; ++q) out[q] = val[slot[q]] * ((kind && pairs[2 * q] == pairs[2 * q + 1]) ? 3.0 : 1.0);
    return XD_OK;
}

}  // namespace xd

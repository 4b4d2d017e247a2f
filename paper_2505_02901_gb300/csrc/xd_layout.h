// xd_layout.h -- the U(1) index layout (Sec. 3.1; Lin's two tables, Sec.
// 5.2).  A word s of N bits with nup ones splits into its top P = N - L bits
// h (prefix) and its low L bits l (postfix).  The block lists its words in
// ascending order, which is ascending h and, within one h, ascending l among
// the L-bit words with m = nup - popcount(h) ones, so
//     index(s) = hi_off[h] + lo_rank[l],
// hi_off[h] = number of block words with a smaller prefix, lo_rank[l] = rank
// of l among the L-bit words of its popcount; lo_list[lo_off[m] + r] is the
// r-th L-bit word with m ones.  Plain C++ without CUDA (the device kernels
// read the same tables; the CPU tests compile this header alone).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace xd {

inline int64_t n_choose_k(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;  // exact at each step
    return r;
}

// Postfix width: a prefix block holds C(L, m) rows, so L bounds the block
// size; the prefix table has 2^(N-L) entries.
inline int choose_L(int N) {
    if (N <= 8) return N;
    int L = (N + 1) / 2;
    if (L > 16) L = 16;
    if (N - L > 24) L = N - 24;
    return L;
}

struct U1Layout {
    int L = 0, P = 0;
    int64_t dim = 0;
    std::vector<int64_t> hi_off;                  // [2^P + 1]
    std::vector<uint32_t> lo_rank, lo_list, lo_off;  // [2^L], [2^L], [L + 2]
};

// The tables at postfix width L; false if they do not add up to C(N, nup)
// (cannot happen for 0 <= nup <= N).
inline bool u1_layout_at(int N, int nup, int L, U1Layout *u) {
    const int P = N - L;
    u->L = L;
    u->P = P;
    const uint64_t nlo = 1ull << L, nhi = 1ull << P;
    u->lo_off.assign(L + 2, 0);
    for (int m = 0; m <= L; ++m) u->lo_off[m + 1] = u->lo_off[m] + (uint32_t)n_choose_k(L, m);
    u->lo_rank.assign(nlo, 0);
    u->lo_list.assign(nlo, 0);
    std::vector<uint32_t> fill(u->lo_off.begin(), u->lo_off.end() - 1);
    for (uint64_t l = 0; l < nlo; ++l) {  // ascending l: ranks in class order
        const int m = __builtin_popcountll(l);
        const uint32_t r = fill[m]++ - u->lo_off[m];
        u->lo_rank[l] = r;
        u->lo_list[u->lo_off[m] + r] = (uint32_t)l;
    }
    u->hi_off.assign(nhi + 1, 0);
    for (uint64_t h = 0; h < nhi; ++h) {
        const int m = nup - __builtin_popcountll(h);
        u->hi_off[h + 1] = u->hi_off[h] + ((m >= 0 && m <= L) ? n_choose_k(L, m) : 0);
    }
    u->dim = u->hi_off[nhi];
    return u->dim == n_choose_k(N, nup);
}

inline bool u1_layout(int N, int nup, U1Layout *u) { return u1_layout_at(N, nup, choose_L(N), u); }

// index of s, or -1 when s is not a word of the block
inline int64_t u1_index(int N, int nup, int L, const std::vector<int64_t> &hi_off,
                        const std::vector<uint32_t> &lo_rank, uint64_t s) {
    if (N < 64 && (s >> N)) return -1;
    if (__builtin_popcountll(s) != nup) return -1;
    return hi_off[s >> L] + lo_rank[s & ((1ull << L) - 1)];
}

// word of index idx, 0 <= idx < dim
inline uint64_t u1_state(int nup, int L, const std::vector<int64_t> &hi_off, const std::vector<uint32_t> &lo_list,
                         const std::vector<uint32_t> &lo_off, int64_t idx) {
    // block: last h with hi_off[h] <= idx
    auto it = std::upper_bound(hi_off.begin(), hi_off.end(), idx);
    const uint64_t h = (uint64_t)(it - hi_off.begin()) - 1;
    const int m = nup - __builtin_popcountll(h);
    const uint32_t l = lo_list[lo_off[m] + (uint32_t)(idx - hi_off[h])];
    return (h << L) | l;
}

// Tables of the block-structured product (one CTA per prefix block).  Bonds
// are postfix (both sites < L), prefix (both >= L: the pair of prefix bits,
// as (a, b, bond) triples) or cross (one site each side: (prefix bit,
// postfix site, bond, slot) quadruples, grouped by prefix bit; csite =
// (prefix bit, first, end) per group; slot = index of the postfix site among
// the distinct cross postfix sites).  Tables are indexed by the class-ordered
// position g of the postfix word l = lo_list[g]:
//   ptab[q 2^L + g] = rank of l with postfix bond q flipped, or maxblk ("no
//   flip" and padding rows; the kernel keeps a zero there),
//   xtab[slot 2^L + g] = rank of l with the slot's postfix site flipped.
struct BlockTables {
    std::vector<int32_t> post, pre, cross, csite;
    std::vector<int> slot_site;
    std::vector<uint16_t> ptab, xtab;
    std::vector<uint32_t> order;  // prefixes with a non-empty block, ascending
    int npost_pad = 0, maxblk = 0;
};

inline void block_tables(int N, int nup, int L, const int32_t *bonds, int nb, const std::vector<uint32_t> &lo_rank,
                         const std::vector<uint32_t> &lo_list, BlockTables *out, bool with_order = true) {
    BlockTables &B = *out;
    const int P = N - L;
    for (int k = 0; k < nb; ++k) {
        int i = bonds[2 * k], j = bonds[2 * k + 1];
        if (i > j) std::swap(i, j);
        if (j < L) {
            B.post.push_back(k);
        } else if (i >= L) {
            B.pre.insert(B.pre.end(), {i - L, j - L, k});
        } else {
            int slot = (int)(std::find(B.slot_site.begin(), B.slot_site.end(), i) - B.slot_site.begin());
            if (slot == (int)B.slot_site.size()) B.slot_site.push_back(i);
            B.cross.insert(B.cross.end(), {j - L, i, k, slot});
        }
    }
    const int nc = (int)B.cross.size() / 4;
    std::vector<int> idx(nc);
    for (int q = 0; q < nc; ++q) idx[q] = q;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return B.cross[4 * a] < B.cross[4 * c]; });
    std::vector<int32_t> sorted;
    for (int q : idx) sorted.insert(sorted.end(), B.cross.begin() + 4 * q, B.cross.begin() + 4 * q + 4);
    B.cross.swap(sorted);
    for (int q = 0; q < nc; ++q)
        if (q == 0 || B.cross[4 * q] != B.cross[4 * (q - 1)]) B.csite.insert(B.csite.end(), {B.cross[4 * q], q, q + 1});
        else B.csite.back() = q + 1;
    const int npost = (int)B.post.size();
    B.npost_pad = (npost + 7) / 8 * 8;
    B.maxblk = (int)n_choose_k(L, L / 2);
    const uint32_t nlo = 1u << L;
    const uint16_t noflip = (uint16_t)B.maxblk;
    B.ptab.assign((size_t)B.npost_pad * nlo, noflip);
    B.xtab.assign(B.slot_site.size() * nlo, 0);
    for (uint32_t g = 0; g < nlo; ++g) {
        const uint32_t l = lo_list[g];
        for (int q = 0; q < npost; ++q) {
            const int i = bonds[2 * B.post[q]], j = bonds[2 * B.post[q] + 1];
            if (((l >> i) & 1) != ((l >> j) & 1)) B.ptab[(size_t)q * nlo + g] = (uint16_t)lo_rank[l ^ (1u << i) ^ (1u << j)];
        }
        for (size_t q = 0; q < B.slot_site.size(); ++q)
            B.xtab[q * nlo + g] = (uint16_t)lo_rank[l ^ (1u << B.slot_site[q])];
    }
    if (with_order)
        for (uint64_t h = 0; h < (1ull << P); ++h) {
            const int m = nup - __builtin_popcountll(h);
            if (m >= 0 && m <= L) B.order.push_back((uint32_t)h);
        }
}

// Work items of the batched FP32 product: kB prefixes of one class m each,
// ascending h within the class; an item is emitted when its class has kB
// prefixes, and each class's last item is padded with `empty`.
inline std::vector<uint32_t> prefix_items(int P, int nup, int L, int kB, uint32_t empty) {
    std::vector<uint32_t> items;
    std::vector<std::vector<uint32_t>> pend(L + 1);
    for (uint64_t h = 0; h < (1ull << P); ++h) {
        const int m = nup - __builtin_popcountll(h);
        if (m < 0 || m > L) continue;
        pend[m].push_back((uint32_t)h);
        if ((int)pend[m].size() == kB) {
            items.insert(items.end(), pend[m].begin(), pend[m].end());
            pend[m].clear();
        }
    }
    for (auto &v : pend)
        if (!v.empty()) {
            items.insert(items.end(), v.begin(), v.end());
            items.insert(items.end(), kB - v.size(), empty);
        }
    return items;
}


// ------------------------------------------------------------ prefix passes
// A prefix bond b (prefix bits a, c) joins block h to block h ^ m_b.  The
// FP64 product treats the prefix bonds in passes: a pass takes the bonds with
// both bits in a window S of at most W prefix bits, so that its flips change
// only the window word of a prefix and a tile over the window words fits in
// shared memory.  choose_passes covers the prefix bonds by such windows,
// greedily: each pass takes, among the candidate W-bit sets, the one that
// covers the most uncovered bonds, ties broken by the fewest bits the
// remaining bonds touch.  Candidates are every window of W consecutive bits
// (whole lattice rows when sites are numbered row by row) and the sets grown
// from every start bit by adding the bit with the most uncovered bonds into
// the set, then the highest degree, then the lowest index.  At most
// max_passes passes; bonds left over join the last one (the kernel would
// then need its window to hold them: callers check every pass bond lies in
// its window).
struct PrefixPass {
    std::vector<int> low;    // the bits placed lowest in the key, ascending
    std::vector<int> bonds;  // indices of the pass's bonds among the prefix triples
};

inline std::vector<PrefixPass> choose_passes(int P, const std::vector<int32_t> &pre, int W, int max_passes) {
    const int n = (int)pre.size() / 3;
    std::vector<char> cov(n, 0);
    std::vector<PrefixPass> out;
    W = std::max(1, std::min(W, P));
    auto remaining_bits = [&](const std::vector<char> &c) {
        uint64_t m = 0;
        for (int q = 0; q < n; ++q)
            if (!c[q]) m |= (1ull << pre[3 * q]) | (1ull << pre[3 * q + 1]);
        return __builtin_popcountll(m);
    };
    int left = n;
    while (left > 0 && (int)out.size() < max_passes) {
        std::vector<int> deg(P, 0);
        for (int q = 0; q < n; ++q)
            if (!cov[q]) {
                ++deg[pre[3 * q]];
                ++deg[pre[3 * q + 1]];
            }
        int best_cnt = -1, best_rem = 1 << 30;
        uint64_t best_set = 0;
        auto consider = [&](uint64_t S) {
            std::vector<char> c2 = cov;
            int cnt = 0;
            for (int q = 0; q < n; ++q)
                if (!cov[q] && ((S >> pre[3 * q]) & 1) && ((S >> pre[3 * q + 1]) & 1)) {
                    c2[q] = 1;
                    ++cnt;
                }
            const int rem = remaining_bits(c2);
            if (cnt > best_cnt || (cnt == best_cnt && rem < best_rem)) {
                best_cnt = cnt;
                best_rem = rem;
                best_set = S;
            }
        };
        for (int s0 = 0; s0 + W <= P; ++s0) consider(((W == 64 ? ~0ull : ((1ull << W) - 1))) << s0);
        for (int start = 0; start < P; ++start) {
            if (deg[start] == 0 && start != 0) continue;
            uint64_t S = 1ull << start;
            for (int k = 1; k < W; ++k) {
                int bv = -1, bin = -1, bdeg = -1;
                for (int v = 0; v < P; ++v) {
                    if ((S >> v) & 1) continue;
                    int in = 0;
                    for (int q = 0; q < n; ++q)
                        if (!cov[q]) {
                            const int a = pre[3 * q], c = pre[3 * q + 1];
                            if ((a == v && ((S >> c) & 1)) || (c == v && ((S >> a) & 1))) ++in;
                        }
                    if (in > bin || (in == bin && deg[v] > bdeg)) {
                        bv = v;
                        bin = in;
                        bdeg = deg[v];
                    }
                }
                if (bv < 0) break;
                S |= 1ull << bv;
            }
            consider(S);
        }
        if (best_cnt <= 0) break;
        PrefixPass ps;
        for (int v = 0; v < P; ++v)
            if ((best_set >> v) & 1) ps.low.push_back(v);
        for (int q = 0; q < n; ++q)
            if (!cov[q] && ((best_set >> pre[3 * q]) & 1) && ((best_set >> pre[3 * q + 1]) & 1)) {
                ps.bonds.push_back(q);
                cov[q] = 1;
                --left;
            }
        out.push_back(ps);
    }
    if (left > 0) {
        if (out.empty()) {
            PrefixPass ps;
            for (int v = 0; v < W; ++v) ps.low.push_back(v);
            out.push_back(ps);
        }
        for (int q = 0; q < n; ++q)
            if (!cov[q]) out.back().bonds.push_back(q);
    }
    return out;
}

// Visiting blocks in the order of a key that places a set of prefix bits
// lowest keeps the blocks reached by flipping those bits close together (in
// L2).  key of prefix h: the bits of `low` (in their order) lowest, then the
// other bits in ascending order.
inline uint32_t pass_key(uint32_t h, const std::vector<int> &low, int P) {
    uint32_t key = 0;
    int k = 0;
    uint32_t used = 0;
    for (int v : low) {
        key |= ((h >> v) & 1u) << k++;
        used |= 1u << v;
    }
    for (int v = 0; v < P; ++v)
        if (!((used >> v) & 1)) key |= ((h >> v) & 1u) << k++;
    return key;
}

// the prefixes with a non-empty block, in ascending key order
inline std::vector<uint32_t> ordered_prefixes(int P, int nup, int L, const std::vector<int> &low) {
    std::vector<std::pair<uint32_t, uint32_t>> kh;
    for (uint64_t h = 0; h < (1ull << P); ++h) {
        const int m = nup - __builtin_popcountll(h);
        if (m >= 0 && m <= L) kh.push_back({pass_key((uint32_t)h, low, P), (uint32_t)h});
    }
    std::sort(kh.begin(), kh.end());
    std::vector<uint32_t> out(kh.size());
    for (size_t i = 0; i < kh.size(); ++i) out[i] = kh[i].second;
    return out;
}

// work items of kB same-class prefixes, emitted in ascending key order of
// their prefixes (each class's last item padded with `empty`)
inline std::vector<uint32_t> ordered_items(int P, int nup, int L, int kB, uint32_t empty, const std::vector<int> &low) {
    std::vector<uint32_t> items;
    std::vector<std::vector<uint32_t>> pend(L + 1);
    for (uint32_t h : ordered_prefixes(P, nup, L, low)) {
        const int m = nup - __builtin_popcountll(h);
        pend[m].push_back(h);
        if ((int)pend[m].size() == kB) {
            items.insert(items.end(), pend[m].begin(), pend[m].end());
            pend[m].clear();
        }
    }
    for (auto &v : pend)
        if (!v.empty()) {
            items.insert(items.end(), v.begin(), v.end());
            items.insert(items.end(), kB - v.size(), empty);
        }
    return items;
}

}  // namespace xd

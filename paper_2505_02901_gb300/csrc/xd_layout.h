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

// false if the tables do not add up to C(N, nup) (cannot happen for 0 <= nup <= N)
inline bool u1_layout(int N, int nup, U1Layout *u) {
    const int L = choose_L(N), P = N - L;
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

}  // namespace xd

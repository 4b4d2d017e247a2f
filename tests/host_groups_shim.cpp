// C entry points over xd_groups.h for the CPU tests (no CUDA).
#include "xd_groups.h"

extern "C" int shim_bond_orbits(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int32_t *orb) {
    return xd::bond_orbits(N, G, perms, bonds, nb, orb);
}

extern "C" int shim_couplings_invariant(int N, int G, const int32_t *perms, const int32_t *bonds, int nb,
                                        const double *J, int *bad_g, int *bad_k) {
    return xd::couplings_invariant(N, G, perms, bonds, nb, J, bad_g, bad_k);
}

// meta[0..5] = nchunk, tx, ty, tnp, cn, cdih; buffers sized by the caller
// (act G*nchunk*256, minrot/amask 256, tg G, tpp G, pm G*nb, cg 2N)
extern "C" void shim_group_tables(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int *meta,
                                  uint64_t *act, uint8_t *minrot, uint8_t *amask, int16_t *tg, int16_t *tpp,
                                  uint64_t *pm, int16_t *cg) {
    xd::GroupTables T;
    xd::group_tables(N, G, perms, bonds, nb, &T);
    meta[0] = T.nchunk; meta[1] = T.tx; meta[2] = T.ty; meta[3] = T.tnp; meta[4] = T.cn; meta[5] = T.cdih;
    for (size_t i = 0; i < T.act.size(); ++i) act[i] = T.act[i];
    for (size_t i = 0; i < T.minrot.size(); ++i) { minrot[i] = T.minrot[i]; amask[i] = T.amask[i]; }
    for (size_t i = 0; i < T.tg.size(); ++i) tg[i] = T.tg[i];
    for (size_t i = 0; i < T.tpp.size(); ++i) tpp[i] = T.tpp[i];
    for (size_t i = 0; i < T.pm.size(); ++i) pm[i] = T.pm[i];
    for (size_t i = 0; i < T.cg.size(); ++i) cg[i] = T.cg[i];
}

// Representative search of xd_orbit.h on n words: rep, |Stab| (pairs of coset
// and translation reaching rep) and the group index of one element reaching
// it, with or without the cut table.  Returns 0 when the group is not a torus
// with Ly <= 8 (or the cut table was asked for and Lx > 7).
#include <vector>
#include "xd_orbit.h"

extern "C" int shim_torus_orbit(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int64_t n,
                                const uint64_t *s, uint64_t *rep, int32_t *cnt, int32_t *u, int use_cut) {
    xd::GroupTables T;
    xd::group_tables(N, G, perms, bonds, nb, &T);
    if (!T.tx || T.ty > 8) return 0;
    std::vector<uint16_t> rowtab(1u << T.tx);
    for (size_t r = 0; r < rowtab.size(); ++r) rowtab[r] = (uint16_t)(T.minrot[r] | (T.amask[r] << 8));
    if (use_cut && T.cut.empty()) return 0;
    const xd::TorusGeo g = xd::torus_geo(T.tx, T.ty, rowtab.data(), use_cut ? T.cut.data() : nullptr);
    auto act = [&](int e, uint64_t w) {
        uint64_t r = 0;
        for (int c = 0; c < T.nchunk; ++c) r |= T.act[((size_t)e * T.nchunk + c) * 256 + ((w >> (8 * c)) & 255)];
        return r;
    };
    const int ncos = T.tnp ? T.tnp : 1;
    for (int64_t i = 0; i < n; ++i) {
        const xd::TorusOrbit o = xd::torus_orbit(g, ncos, [&](int k) { return k ? act(T.tpp[k], s[i]) : s[i]; });
        rep[i] = o.rep;
        cnt[i] = o.cnt;
        u[i] = T.tg[(size_t)o.k * N + (o.q & 7) + T.tx * (o.q >> 3)];
    }
    return 1;
}

// Incremental top step (xd_orbit.h): the row state of s refreshed in the rows
// of sites i and j against the top step of s ^ (bit i | bit j) computed from
// the word; returns the number of words where top row or candidates differ.
extern "C" int64_t shim_top_rows_mismatch(int N, int G, const int32_t *perms, const int32_t *bonds, int nb,
                                          int64_t n, const uint64_t *s, const int32_t *ij) {
    xd::GroupTables T;
    xd::group_tables(N, G, perms, bonds, nb, &T);
    if (!T.tx || T.ty > 8) return -1;
    if (T.tx > 7) return -2;  // row states hold rows of at most 7 sites
    std::vector<uint16_t> rowtab(1u << T.tx);
    for (size_t r = 0; r < rowtab.size(); ++r) rowtab[r] = (uint16_t)(T.minrot[r] | (T.amask[r] << 8));
    const xd::TorusGeo g = xd::torus_geo(T.tx, T.ty, rowtab.data());
    int64_t bad = 0;
    for (int64_t q = 0; q < n; ++q) {
        uint64_t PM, PA;
        xd::torus_rows(g, s[q], PM, PA);
        const int i = ij[2 * q], j = ij[2 * q + 1];
        const uint64_t w = s[q] ^ (1ull << i) ^ (1ull << j);
        xd::torus_rows_set(g, PM, PA, w, i / T.tx);
        xd::torus_rows_set(g, PM, PA, w, j / T.tx);
        uint32_t t1, t2;
        const uint64_t M1 = xd::torus_top_rows(g, PM, PA, &t1);
        const uint64_t M2 = xd::torus_top(g, w, &t2);
        bad += (t1 != t2 || M1 != M2);
    }
    return bad;
}

// The top step from the three smallest rows (xd_orbit.h) against the top
// step of s ^ (bit i | bit j) from the word; number of differing words.
extern "C" int64_t shim_top3_mismatch(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int64_t n,
                                      const uint64_t *s, const int32_t *ij) {
    xd::GroupTables T;
    xd::group_tables(N, G, perms, bonds, nb, &T);
    if (!T.tx || T.ty > 8) return -1;
    if (T.tx > 7) return -2;
    std::vector<uint16_t> rowtab(1u << T.tx);
    for (size_t r = 0; r < rowtab.size(); ++r) rowtab[r] = (uint16_t)(T.minrot[r] | (T.amask[r] << 8));
    const xd::TorusGeo g = xd::torus_geo(T.tx, T.ty, rowtab.data());
    int64_t bad = 0;
    for (int64_t q = 0; q < n; ++q) {
        xd::RowTop3 t;
        xd::torus_top3(g, s[q], t);
        const int i = ij[2 * q], j = ij[2 * q + 1];
        const uint64_t w = s[q] ^ (1ull << i) ^ (1ull << j);
        uint32_t t1, t2;
        const uint64_t M1 = xd::torus_top_flip(g, t, w, i / T.tx, j / T.tx, &t1);
        const uint64_t M2 = xd::torus_top(g, w, &t2);
        bad += (t1 != t2 || M1 != M2);
    }
    return bad;
}

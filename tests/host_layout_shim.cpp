// C entry points over xd_layout.h for the CPU tests (no CUDA).
#include "xd_layout.h"

static xd::U1Layout g_lay;
static int g_N = 0, g_nup = 0;

extern "C" int shim_u1_build(int N, int nup, long long *dim, int *L) {
    g_N = N;
    g_nup = nup;
    const bool ok = xd::u1_layout(N, nup, &g_lay);
    *dim = g_lay.dim;
    *L = g_lay.L;
    return ok ? 1 : 0;
}

extern "C" long long shim_u1_index(unsigned long long s) {
    return xd::u1_index(g_N, g_nup, g_lay.L, g_lay.hi_off, g_lay.lo_rank, s);
}

extern "C" unsigned long long shim_u1_state(long long idx) {
    return xd::u1_state(g_nup, g_lay.L, g_lay.hi_off, g_lay.lo_list, g_lay.lo_off, idx);
}

static xd::BlockTables g_blk;

// sizes: L, npost, npre, ncross, ncsite, nslot, npost_pad, maxblk, norder
extern "C" void shim_block_build_at(int N, int nup, int L, const int32_t *bonds, int nb, int *sizes) {
    g_N = N;
    g_nup = nup;
    xd::u1_layout_at(N, nup, L > 0 ? L : xd::choose_L(N), &g_lay);
    g_blk = xd::BlockTables();
    xd::block_tables(N, nup, g_lay.L, bonds, nb, g_lay.lo_rank, g_lay.lo_list, &g_blk);
    const int s[9] = {g_lay.L, (int)g_blk.post.size(), (int)g_blk.pre.size() / 3, (int)g_blk.cross.size() / 4,
                      (int)g_blk.csite.size() / 3, (int)g_blk.slot_site.size(), g_blk.npost_pad, g_blk.maxblk,
                      (int)g_blk.order.size()};
    for (int i = 0; i < 9; ++i) sizes[i] = s[i];
}
extern "C" const int64_t *shim_hi_off() { return g_lay.hi_off.data(); }
extern "C" const uint32_t *shim_lo_rank() { return g_lay.lo_rank.data(); }
extern "C" const uint32_t *shim_lo_list() { return g_lay.lo_list.data(); }
extern "C" const uint32_t *shim_lo_off() { return g_lay.lo_off.data(); }
extern "C" const int32_t *shim_post() { return g_blk.post.data(); }
extern "C" const int32_t *shim_pre() { return g_blk.pre.data(); }
extern "C" const int32_t *shim_cross() { return g_blk.cross.data(); }
extern "C" const int32_t *shim_csite() { return g_blk.csite.data(); }
extern "C" const uint16_t *shim_ptab() { return g_blk.ptab.data(); }
extern "C" const uint16_t *shim_xtab() { return g_blk.xtab.data(); }
extern "C" const uint32_t *shim_order() { return g_blk.order.data(); }

extern "C" void shim_block_build(int N, int nup, const int32_t *bonds, int nb, int *sizes) {
    shim_block_build_at(N, nup, 0, bonds, nb, sizes);
}

extern "C" long long shim_items(int P, int nup, int L, int kB, uint32_t empty, uint32_t *out, long long cap) {
    const std::vector<uint32_t> v = xd::prefix_items(P, nup, L, kB, empty);
    for (size_t i = 0; i < v.size() && (long long)i < cap; ++i) out[i] = v[i];
    return (long long)v.size();
}

// prefix passes: returns the number of passes; for pass p, low bits and
// bonds (indices into the prefix triples) are written to the out arrays
static std::vector<xd::PrefixPass> g_passes;
extern "C" int shim_choose_passes(int P, const int32_t *pre, int npre, int W, int max_passes) {
    g_passes = xd::choose_passes(P, std::vector<int32_t>(pre, pre + 3 * npre), W, max_passes);
    return (int)g_passes.size();
}
extern "C" int shim_pass_low(int p, int32_t *out) {
    for (size_t i = 0; i < g_passes[p].low.size(); ++i) out[i] = g_passes[p].low[i];
    return (int)g_passes[p].low.size();
}
extern "C" int shim_pass_bonds(int p, int32_t *out) {
    for (size_t i = 0; i < g_passes[p].bonds.size(); ++i) out[i] = g_passes[p].bonds[i];
    return (int)g_passes[p].bonds.size();
}
extern "C" long long shim_ordered_items(int P, int nup, int L, int kB, uint32_t empty, const int32_t *low, int nlow,
                                        uint32_t *out, long long cap) {
    const std::vector<uint32_t> v = xd::ordered_items(P, nup, L, kB, empty, std::vector<int>(low, low + nlow));
    for (size_t i = 0; i < v.size() && (long long)i < cap; ++i) out[i] = v[i];
    return (long long)v.size();
}

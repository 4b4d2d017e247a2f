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

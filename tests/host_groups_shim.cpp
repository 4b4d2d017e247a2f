// C entry points over xd_groups.h for the CPU tests (no CUDA).
#include "xd_groups.h"

extern "C" int shim_bond_orbits(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int32_t *orb) {
    return xd::bond_orbits(N, G, perms, bonds, nb, orb);
}

extern "C" int shim_couplings_invariant(int N, int G, const int32_t *perms, const int32_t *bonds, int nb,
                                        const double *J, int *bad_g, int *bad_k) {
    return xd::couplings_invariant(N, G, perms, bonds, nb, J, bad_g, bad_k);
}

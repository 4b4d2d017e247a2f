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

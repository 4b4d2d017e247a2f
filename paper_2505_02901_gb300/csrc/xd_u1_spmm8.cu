// xd_u1_spmm8.cu -- FP32 Y = H X for eight right-hand sides on a large U(1)
// block (X, Y row-major [dim][8]; the multi-vector apply of Sec. 5.1).
//
// Same decomposition as the one-vector product of xd_u1_spmm.cu (the
// prefix/postfix view of Sec. 5.3, H = H_post + H_pre + H_cross), with the
// eight columns of one prefix block in the place of eight blocks: a CTA
// takes one prefix block h at a time and stages its rows (32 bytes each, the
// eight values of a row) in shared memory.
//   * H_post: one target rank per row and postfix bond serves eight values.
//   * H_pre: the rows of the neighbour block h ^ m_b are read in place, 32
//     bytes per row, coalesced across the CTA's threads.
//   * H_cross: for every cross prefix site a the neighbour block h ^ 2^a is
//     staged (16-byte copies, double-buffered); a row flips with bond (a, j)
//     when bit j of its postfix word differs from bit a of h, the same test
//     for all eight columns.
// Rows are written once (pull form), no atomics; all sums in FP32.

#include <algorithm>
#include <vector>

#include "xd_spmm8.cuh"

namespace xd {

using namespace sp8;

namespace {

template <int L>
__global__ void __launch_bounds__(kT8, 2) k_spmm8(Sp8Params p, const float *__restrict__ x,
                                              float *__restrict__ y) {
    extern __shared__ __align__(128) unsigned char smem[];
    tables<L>(p, smem);
    for (int64_t t = blockIdx.x; t < p.nprefix; t += gridDim.x) {
        const uint32_t h = __ldg(p.items + t);
        if (h == kEmpty8) continue;  // the same for every thread of the CTA
        block<L>(p, smem, h, x, y);
    }
}

template <int L>
xd_status launch_spmm8(const xd_ham_s *h, const float *x, float *y, cudaStream_t st) {
    Sp8Params p;
    sp8_params(h, &p);
    const Sp8Smem lay(p, Sp8Geo<L>::maxblk);
    auto kern = k_spmm8<L>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT8, lay.total));
    if (per_sm < 1) {
        set_error("eight-vector product: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    grid_for(1, 1, 1);
    const int grid = (int)std::min<int64_t>(p.nprefix, (int64_t)g_num_sms * per_sm);
    kern<<<grid, kT8, lay.total, st>>>(p, x, y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

}  // namespace

void sp8_params(const xd_ham_s *h, Sp8Params *out) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    Sp8Params &p = *out;
    p.nup = b->nup;
    p.hi_off = s.d_hi_off;
    p.lo_off = s.d_lo_off;
    p.lo_list = s.d_lo_list;
    p.items = s.d_items;
    p.nprefix = s.nitems * 8;
    p.ptab = s.d_ptab;
    p.npost_pad = s.npost_pad;
    p.xtab = s.d_xtab;
    p.dpost = h->d_sp_dpost;
    p.pcsr_off = s.d_pcsr_off;
    p.pcsr = s.d_pcsr;
    p.maxpa = s.maxpa;
    p.pre = s.d_pre;
    p.npre = s.npre;
    p.cross = s.d_cross;
    p.ncross = s.ncross;
    p.csite = s.d_csite;
    p.ncsite = s.ncsite;
    p.jhalf = h->d_sp_jhalf;
    p.postid = s.d_postid;
    p.nb = b->nb;
    p.jcross = h->sp_jcross;
}

bool spmm8_usable(const xd_ham_s *h, const void *x, const void *y) {
    return h->b->spmm.ok && !h->b->sym && ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0;
}

xd_status spmm8_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    switch (h->b->spmm.L) {
        case 10: return launch_spmm8<10>(h, (const float *)x, (float *)y, st);
        case 11: return launch_spmm8<11>(h, (const float *)x, (float *)y, st);
        case 12: return launch_spmm8<12>(h, (const float *)x, (float *)y, st);
        default:
            set_error("eight-vector product: postfix length %d not supported", h->b->spmm.L);
            return XD_ERANGE;
    }
}

}  // namespace xd

// xd_u1_block.cu -- block-structured y = H x on large U(1) blocks.
//
// Same product as xd_u1.cu (Eq. 1, pull form), organised around the
// prefix/postfix split of the index layout.  XDiag distributes states by
// prefix and applies postfix-only terms locally (Sec. 5.3); here one CTA
// owns one prefix block h (the C(L, m) consecutive rows sharing the prefix,
// m = nup - popcount(h)) and the bonds fall into three kinds:
//   postfix bonds (both sites < L): the flipped state stays in block h; its
//       rank inside the block comes from a bond-major target table indexed by
//       the in-class rank of the row (so a warp reads consecutive entries),
//       and x of the whole block is staged in shared memory, so these
//       gathers are shared-memory loads;
//   prefix bonds (both sites >= L): the flip maps block h to block h ^ m_b
//       with the same in-block rank, so row i reads x[off(h') + i]: one
//       coalesced stream per active bond, decided once per block;
//   cross bonds (one site each side): the flip changes the prefix bit a (one
//       neighbour block per prefix site a) and one postfix bit j of l.  The
//       neighbour block of each cross site is copied into shared memory with
//       cp.async (double buffered: the copy of the next neighbour overlaps
//       the gathers from the current one); the rank of l ^ 2^j in its class
//       comes from a per-site table indexed by the row's in-class rank.
// Each thread owns K rows of the block (i = tid + k * 1024) and keeps their
// accumulators in registers across the three phases.  The diagonal is
// d_pre(h) + d_post(l) + the cross-bond terms.  Prefix blocks are walked in
// ascending order (static round robin), so the blocks reached by flips on
// low prefix bits are still in L2.

#include <algorithm>
#include <vector>

#include "xd_internal.cuh"
#include "xd_layout.h"

namespace xd {

namespace {

template <typename T>
struct PreEnt {
    const T *src;   // x + first row of the neighbour block
    T coef;         // J/2
};

struct BlkParams {
    U1View u;
    const uint32_t *order;  // non-empty prefixes, ascending
    int64_t nblk;
    const uint16_t *ptab;   // [npost_pad][2^L]: rank of l ^ m_b in class, maxblk = no flip
    const uint16_t *xtab;   // [nslot][2^L]: rank of l ^ 2^j_slot in its class
    const double *dpost;    // [2^L]: postfix diagonal, by class-ordered position
    const int32_t *post;    // [npost] bond ids
    int npost, npost_pad;   // postfix bonds, padded to a multiple of 8 (dummy rows never flip)
    const double *J;        // [nb]
    const int32_t *pre;     // [npre][3]: prefix bit a, prefix bit b, bond id
    int npre;
    const int32_t *cross;   // [ncross][4]: prefix bit, postfix site, bond id, slot (grouped by prefix bit)
    int ncross;
    const int32_t *csite;   // [ncsite][3]: prefix bit a, first cross bond, end cross bond
    int ncsite;
    int nb;
    int maxblk;
    double jcross;          // sum over cross bonds of J/4
};

constexpr int kBT = 1024;   // threads per CTA

template <int L>
struct Geo {
    static constexpr uint32_t nlo = 1u << L;
    static constexpr int maxblk = L == 16 ? 12870 : L == 15 ? 6435 : L == 14 ? 3432 : L == 13 ? 1716
                                : L == 12 ? 924 : L == 11 ? 462 : 252;
    static constexpr int K = (maxblk + kBT - 1) / kBT;  // rows per thread
};

template <typename T>
struct SmemLayout {
    size_t xs, nbuf, pc, cc, cmeta, pre, site, total;
    __host__ __device__ SmemLayout(const BlkParams &p, int nbufs) {
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;
        o += (size_t)(p.maxblk + 1) * sizeof(T);  // + a zero slot for "no flip"
        al(16);
        nbuf = o;
        o += (size_t)nbufs * p.maxblk * sizeof(T);
        al(16);
        pc = o;
        o += (size_t)p.npost_pad * sizeof(T);
        al(16);
        cc = o;
        o += (size_t)p.ncross * sizeof(T);
        al(16);
        cmeta = o;
        o += (size_t)p.ncross * sizeof(uint32_t);
        al(16);
        pre = o;
        o += (size_t)p.npre * sizeof(PreEnt<T>);
        al(16);
        site = o;
        o += (size_t)p.ncsite * sizeof(int64_t) * 2;
        al(16);
        total = o;
    }
};

__device__ __forceinline__ void cp_async(void *smem_dst, const void *gsrc, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T>
__device__ __forceinline__ void stage(T *dst, const T *src, int n) {
    for (int i = threadIdx.x; i < n; i += kBT) cp_async(dst + i, src + i, (int)sizeof(T));
    cp_commit();
}

template <typename T, int L, int NBUF>
__global__ void __launch_bounds__(kBT) k_block_apply(BlkParams p, const T *__restrict__ x,
                                                     T *__restrict__ y) {
    using G = Geo<L>;
    constexpr uint32_t nlo = G::nlo;
    constexpr int K = G::K;
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout<T> lay(p, NBUF);
    T *xs = (T *)(smem + lay.xs);
    T *nbuf = (T *)(smem + lay.nbuf);
    T *pc = (T *)(smem + lay.pc);
    T *cc = (T *)(smem + lay.cc);
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);
    PreEnt<T> *pl = (PreEnt<T> *)(smem + lay.pre);
    int64_t *site = (int64_t *)(smem + lay.site);  // [ncsite][2]: neighbour offset, (n << 1) | req
    __shared__ int sh_npa;
    __shared__ double sh_dpre;

    const U1View &u = p.u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < p.npost_pad; k += kBT) pc[k] = k < p.npost ? (T)(0.5 * p.J[p.post[k]]) : T(0);
    for (int q = tid; q < p.ncross; q += kBT) {
        cc[q] = (T)(0.5 * p.J[p.cross[4 * q + 2]]);
        cmeta[q] = (uint32_t)p.cross[4 * q + 1] | ((uint32_t)p.cross[4 * q + 3] << 8);
    }

    for (int64_t t = blockIdx.x; t < p.nblk; t += gridDim.x) {
        const uint64_t h = p.order[t];
        const int m = u.nup - __popcll(h);
        const uint32_t l0 = __ldg(u.lo_off + m);
        const int n = (int)(__ldg(u.lo_off + m + 1) - l0);
        const int64_t off = __ldg(u.hi_off + h);
        __syncthreads();  // previous block done with shared memory
        stage(xs, x + off, n);
        if (tid == 0) xs[p.maxblk] = T(0);
        if (warp == 0) {
            // active prefix bonds (ballot compaction) and the prefix diagonal
            int cnt = 0;
            double dpre = 0.0;
            for (int base = 0; base < p.npre; base += 32) {
                const int q = base + lane;
                bool act = false;
                int a = 0, b = 0;
                double Jq = 0.0;
                if (q < p.npre) {
                    a = p.pre[3 * q];
                    b = p.pre[3 * q + 1];
                    Jq = p.J[p.pre[3 * q + 2]];
                    act = ((h >> a) & 1) != ((h >> b) & 1);
                    dpre += act ? -0.25 * Jq : 0.25 * Jq;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, act);
                if (act) {
                    const int pos = cnt + __popc(bal & ((1u << lane) - 1));
                    PreEnt<T> e;
                    e.src = x + __ldg(u.hi_off + (h ^ ((1ull << a) | (1ull << b))));
                    e.coef = (T)(0.5 * Jq);
                    pl[pos] = e;
                }
                cnt += __popc(bal);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dpre += __shfl_xor_sync(0xffffffffu, dpre, o);
            if (lane == 0) {
                sh_npa = cnt;
                sh_dpre = dpre + p.jcross;
            }
        } else if (warp == 1) {
            for (int c = lane; c < p.ncsite; c += 32) {
                const int a = p.csite[3 * c];
                const int hb = (int)((h >> a) & 1);
                const int mn = hb ? m + 1 : m - 1;  // class of the neighbour block
                const int nn = (mn >= 0 && mn <= L) ? (int)(__ldg(u.lo_off + mn + 1) - __ldg(u.lo_off + mn)) : 0;
                site[2 * c] = __ldg(u.hi_off + (h ^ (1ull << a)));
                site[2 * c + 1] = ((int64_t)nn << 1) | (int64_t)(1 - hb);
            }
        }
        __syncthreads();
        // the first cross neighbour copy overlaps the postfix and prefix phases
        if (p.ncsite > 0) stage(nbuf, x + site[0], (int)(site[1] >> 1));
        if (p.ncsite > 0) cp_wait<1>(); else cp_wait<0>();
        __syncthreads();  // xs complete

        T acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = T(0);
        // postfix bonds: target ranks from the bond-major table (compile-time
        // stride; "no flip" points at the zero slot), x from xs, branch free
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = tid + k * kBT;
            if (i < n) {
                const uint16_t *pt = p.ptab + l0 + i;
                const T *pcb = pc;
                T a = T(0);
#pragma unroll 1
                for (int b0 = 0; b0 < p.npost_pad; b0 += 8, pt += 8 * nlo, pcb += 8) {
                    uint32_t r[8];
#pragma unroll
                    for (int v = 0; v < 8; ++v) r[v] = __ldg(pt + v * nlo);
#pragma unroll
                    for (int v = 0; v < 8; ++v) a += pcb[v] * xs[r[v]];
                }
                acc[k] += a;
            }
        }
        // prefix bonds: coalesced streams from the neighbour blocks
        {
            const int npa = sh_npa;
#pragma unroll 1
            for (int q = 0; q < npa; ++q) {
                const PreEnt<T> e = pl[q];
                T v[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = tid + k * kBT;
                    v[k] = i < n ? __ldg(e.src + i) : T(0);
                }
#pragma unroll
                for (int k = 0; k < K; ++k) acc[k] += e.coef * v[k];
            }
        }
        // cross bonds: one staged neighbour block per prefix site; a flip adds
        // J/2 (x_target - x_row), which also takes J/2 off the diagonal
        for (int c = 0; c < p.ncsite; ++c) {
            T *buf = nbuf + (NBUF == 2 ? (c & 1) : 0) * p.maxblk;
            if (NBUF == 2) {
                if (c + 1 < p.ncsite) {
                    __syncthreads();  // the other buffer is free (its site finished)
                    stage(nbuf + ((c + 1) & 1) * p.maxblk, x + site[2 * (c + 1)], (int)(site[2 * c + 3] >> 1));
                    cp_wait<1>();
                } else {
                    cp_wait<0>();
                }
            } else {
                if (c > 0) {
                    __syncthreads();
                    stage(buf, x + site[2 * c], (int)(site[2 * c + 1] >> 1));
                }
                cp_wait<0>();
            }
            __syncthreads();  // buffer of site c complete
            const uint32_t req = (uint32_t)(site[2 * c + 1] & 1);
            const int q0 = p.csite[3 * c + 1], q1 = p.csite[3 * c + 2];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = tid + k * kBT;
                if (i < n) {
                    const uint32_t l = __ldg(u.lo_list + l0 + i);
                    const T xi = xs[i];
                    T a = T(0);
#pragma unroll 1
                    for (int q = q0; q < q1; ++q) {
                        const uint32_t meta = cmeta[q];
                        // rank of l ^ 2^j in its class: inside the buffer even
                        // when the bond does not flip; the select drops that value
                        const bool f = ((l >> (meta & 31u)) & 1u) == req;
                        if constexpr (sizeof(T) == 8) {
                            // double: the FP64 pipe is the scarce one, branch instead
                            if (f) a += cc[q] * (buf[__ldg(p.xtab + (size_t)(meta >> 8) * nlo + (l0 + i))] - xi);
                        } else {
                            const uint32_t r2 = __ldg(p.xtab + (size_t)(meta >> 8) * nlo + (l0 + i));
                            const T t = cc[q] * (buf[r2] - xi);
                            a += f ? t : T(0);
                        }
                    }
                    acc[k] += a;
                }
            }
        }
        const T dpre = (T)sh_dpre;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int i = tid + k * kBT;
            if (i < n) y[off + i] = (dpre + (T)__ldg(p.dpost + l0 + i)) * xs[i] + acc[k];
        }
    }
}

}  // namespace

// ------------------------------------------------------------ host side

bool block_layout_wanted(const xd_basis_s *b) {
    if (b->sym || b->N < 20 || b->L < 10) return false;
    int ncross = 0;
    for (const Bond &bd : b->bonds) {
        int i = std::min(bd.i, bd.j), j = std::max(bd.i, bd.j);
        ncross += (i < b->L && j >= b->L);
    }
    return ncross <= 1024 && b->L >= 10 && b->L <= 16;
}

xd_status block_layout_build(xd_basis_s *b) {
    const int L = b->L, nup = b->nup;
    BlockLayoutHost &bl = b->blk;
    BlockTables T;
    block_tables(b->N, nup, L, (const int32_t *)b->bonds.data(), b->nb, b->h_lo_rank, b->h_lo_list, &T);
    bl.ncsite = (int)T.csite.size() / 3;
    bl.npre = (int)T.pre.size() / 3;
    bl.ncross = (int)T.cross.size() / 4;
    bl.npost = (int)T.post.size();
    bl.npost_pad = T.npost_pad;
    bl.post.assign(T.post.begin(), T.post.end());
    bl.nblk = (int64_t)T.order.size();
    bl.maxblk = T.maxblk;
    const std::vector<uint32_t> &order = T.order;
    const std::vector<int32_t> &post = T.post, &pre = T.pre, &cross = T.cross, &csite = T.csite;
    const std::vector<uint16_t> &ptab = T.ptab, &xtab = T.xtab;
    auto up = [](auto **dst, const auto &v) -> xd_status {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        XD_CUDA(dev_malloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(E)));
        if (!v.empty()) XD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
        return XD_OK;
    };
    XD_TRY(up(&bl.d_order, order));
    XD_TRY(up(&bl.d_ptab, ptab));
    XD_TRY(up(&bl.d_xtab, xtab));
    XD_TRY(up(&bl.d_postid, post));
    XD_TRY(up(&bl.d_pre, pre));
    XD_TRY(up(&bl.d_cross, cross));
    XD_TRY(up(&bl.d_csite, csite));
    bl.ok = true;
    return XD_OK;
}

void block_layout_free(xd_basis_s *b) {
    BlockLayoutHost &bl = b->blk;
    cudaFree(bl.d_order);
    cudaFree(bl.d_ptab);
    cudaFree(bl.d_xtab);
    cudaFree(bl.d_postid);
    cudaFree(bl.d_pre);
    cudaFree(bl.d_cross);
    cudaFree(bl.d_csite);
    bl = BlockLayoutHost();
}

// d_post[g] = sum over postfix bonds of J/4 (+1 equal spins, -1 opposite)
// for the postfix word at class-ordered position g.
xd_status block_ham_tables(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const uint32_t nlo = 1u << b->L;
    std::vector<double> dpost(nlo, 0.0);
    for (uint32_t g = 0; g < nlo; ++g) {
        const uint32_t l = b->h_lo_list[g];
        double d = 0.0;
        for (int k : b->blk.post) {
            int i = b->bonds[k].i, j = b->bonds[k].j;
            d += (((l >> i) & 1) == ((l >> j) & 1) ? 0.25 : -0.25) * h->J[k];
        }
        dpost[g] = d;
    }
    if (!h->d_dpost) XD_CUDA(dev_malloc((void **)&h->d_dpost, nlo * sizeof(double)));
    XD_CUDA(cudaMemcpy(h->d_dpost, dpost.data(), nlo * sizeof(double), cudaMemcpyHostToDevice));
    return XD_OK;
}

template <typename T, int L, int NBUF>
static xd_status launch_block(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const BlockLayoutHost &bl = b->blk;
    BlkParams p;
    p.u = b->u1view();
    p.order = bl.d_order;
    p.nblk = bl.nblk;
    p.ptab = bl.d_ptab;
    p.xtab = bl.d_xtab;
    p.post = bl.d_postid;
    p.npost = bl.npost;
    p.npost_pad = bl.npost_pad;
    p.J = h->d_J;
    p.dpost = h->d_dpost;
    double q = 0.0;
    for (int k = 0; k < b->nb; ++k) {
        int i = std::min(b->bonds[k].i, b->bonds[k].j), j = std::max(b->bonds[k].i, b->bonds[k].j);
        if (i < b->L && j >= b->L) q += h->J[k];
    }
    p.jcross = 0.25 * q;
    p.pre = bl.d_pre;
    p.npre = bl.npre;
    p.cross = bl.d_cross;
    p.ncross = bl.ncross;
    p.csite = bl.d_csite;
    p.ncsite = bl.ncsite;
    p.nb = b->nb;
    p.maxblk = Geo<L>::maxblk;
    const SmemLayout<T> lay(p, NBUF);
    auto kern = k_block_apply<T, L, NBUF>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBT, lay.total));
    if (per_sm < 1) {
        set_error("block kernel: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    grid_for(1, 1, 1);
    const int grid = (int)std::min<int64_t>(p.nblk, (int64_t)g_num_sms * per_sm);
    kern<<<grid, kBT, lay.total, st>>>(p, (const T *)x, (T *)y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

template <typename T, int L>
static xd_status launch_nb(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    // two neighbour buffers when two CTAs with three block buffers each fit
    const size_t blk = (size_t)Geo<L>::maxblk * sizeof(T);
    if (6 * blk <= 220 * 1024) return launch_block<T, L, 2>(h, x, y, st);
    return launch_block<T, L, 1>(h, x, y, st);
}

template <typename T>
static xd_status launch_L(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    switch (h->b->L) {
        case 10: return launch_nb<T, 10>(h, x, y, st);
        case 11: return launch_nb<T, 11>(h, x, y, st);
        case 12: return launch_nb<T, 12>(h, x, y, st);
        case 13: return launch_nb<T, 13>(h, x, y, st);
        case 14: return launch_nb<T, 14>(h, x, y, st);
        case 15: return launch_nb<T, 15>(h, x, y, st);
        default: return launch_nb<T, 16>(h, x, y, st);
    }
}

xd_status block_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt, cudaStream_t st) {
    if (dt == XD_F64) return launch_L<double>(h, x, y, st);
    return launch_L<float>(h, x, y, st);
}

}  // namespace xd

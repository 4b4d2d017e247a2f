// xd_u1_spmm.cu -- FP32 y = H x on large U(1) blocks as a batched sparse
// product over prefix blocks.
//
// With the prefix/postfix split of the index layout (Sec. 5.2 two tables,
// Sec. 5.3 prefix/postfix view), H = H_post + H_pre + H_cross:
//   * H_post (both sites below L) acts on the postfix rank only, with the
//     same sparse matrix for every prefix block of one class m.  A CTA takes
//     kB prefix blocks of one class, stages their x transposed in shared
//     memory (xs[row][block]) and, per row and postfix bond, reads one target
//     rank and two 16-byte rows of xs: one index serves kB blocks.
//   * H_pre (both sites at or above L) maps block h to block h ^ m_b with the
//     same in-block rank: coalesced streams from the neighbour blocks, whose
//     row offsets are precomputed per prefix (CSR over prefixes).
//   * H_cross (one site each side) flips one prefix bit a and one postfix
//     bit j: for every cross prefix site the kB neighbour blocks are staged
//     transposed with cp.async, and the rank of l ^ 2^j in its class comes
//     from a per-site table; blocks for which the bond does not flip get a
//     zero coefficient.
// Rows are written once (pull form), no atomics; all sums in FP32.

#include <algorithm>
#include <vector>

#include "xd_internal.cuh"
#include "xd_layout.h"

namespace xd {

namespace {

constexpr int kB = 8;                 // prefix blocks per work item
constexpr int kT = 512;               // threads per CTA
constexpr uint32_t kEmpty = 0xffffffffu;

template <int L>
struct SpGeo {
    static constexpr uint32_t nlo = 1u << L;
    static constexpr int maxblk = L == 13 ? 1716 : L == 12 ? 924 : L == 11 ? 462 : 252;
    static constexpr int K = (maxblk + kT - 1) / kT;  // rows per thread
};

struct SpParams {
    int nup;
    const int64_t *hi_off;      // [2^P + 1]
    const uint32_t *lo_off;     // [L + 2]
    const uint32_t *lo_list;    // [2^L]
    const uint32_t *items;      // [nitems][kB]
    int64_t nitems;
    const uint16_t *ptab;       // [npost_pad][2^L], "no flip" = maxblk (zero row)
    int npost_pad;
    const uint16_t *xtab;       // [nslot][2^L]
    const float *dpost;         // [2^L] postfix diagonal by class position
    const int64_t *pcsr_off;    // [2^P + 1] active prefix bonds per prefix
    const uint64_t *pcsr;       // (neighbour block row offset << 12) | bond id
    int maxpa;                  // most active prefix bonds of any prefix
    const int32_t *pre;         // [npre][3] prefix bit a, prefix bit b, bond id
    int npre;
    const int32_t *cross;       // [ncross][4] prefix bit, postfix site, bond id, slot
    int ncross;
    const int32_t *csite;       // [ncsite][3] prefix bit, first, end (cross grouped by site)
    int ncsite;
    const float *jhalf;         // [nb] J/2
    const uint16_t *postid;     // [npost_pad] bond id (0 for padding)
    int nb;
    float jcross;               // sum over cross bonds of J/4
};

constexpr int kPB = 16;  // prefix bonds per step of the prefix streams
__host__ __device__ inline int pad_pa(int maxpa) { return (maxpa + kPB - 1) / kPB * kPB; }

struct SpSmem {
    size_t xs, nb, jh, pc, pl, plc, cmeta, cc, rqm, noff, nn, total;
    __host__ __device__ SpSmem(const SpParams &p, int maxblk) {
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;
        o += (size_t)(maxblk + 1) * kB * sizeof(float);
        al(16);
        nb = o;  // two staging buffers for cross sites
        o += 2 * (size_t)(maxblk + 1) * kB * sizeof(float);
        al(16);
        jh = o;
        o += (size_t)p.nb * sizeof(float);
        al(16);
        pc = o;
        o += (size_t)p.npost_pad * sizeof(float);
        al(16);
        pl = o;
        o += (size_t)kB * p.maxpa * sizeof(uint64_t);
        al(16);
        plc = o;  // coefficients of the listed bonds, zero-padded to kPB
        o += (size_t)kB * pad_pa(p.maxpa) * sizeof(float);
        al(16);
        cmeta = o;
        o += (size_t)p.ncross * sizeof(uint32_t);
        al(16);
        cc = o;
        o += (size_t)p.ncross * sizeof(float);
        al(16);
        rqm = o;
        o += (size_t)p.ncsite * sizeof(uint32_t);
        al(16);
        noff = o;
        o += (size_t)p.ncsite * kB * sizeof(int64_t);
        al(16);
        nn = o;
        o += (size_t)p.ncsite * kB * sizeof(int);
        al(16);
        total = o;
    }
};

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Transposed rows are 32 bytes; the halves of rows with bit 2 set are
// swapped so that 16-byte loads of eight consecutive rows hit distinct banks.
__device__ __forceinline__ int swz(int r, int k) { return r * kB + (k ^ (((r >> 2) & 1) << 2)); }

__device__ __forceinline__ void row8(const float *base, int r, float4 &lo, float4 &hi) {
    const int s = ((r >> 2) & 1) << 2;
    lo = *(const float4 *)(base + r * kB + s);
    hi = *(const float4 *)(base + r * kB + (4 - s));
}

__device__ __forceinline__ void fma8(float (&a)[kB], float c, const float *base, int r) {
    float4 lo, hi;
    row8(base, r, lo, hi);
    a[0] = fmaf(c, lo.x, a[0]); a[1] = fmaf(c, lo.y, a[1]);
    a[2] = fmaf(c, lo.z, a[2]); a[3] = fmaf(c, lo.w, a[3]);
    a[4] = fmaf(c, hi.x, a[4]); a[5] = fmaf(c, hi.y, a[5]);
    a[6] = fmaf(c, hi.z, a[6]); a[7] = fmaf(c, hi.w, a[7]);
}

template <int L>
__global__ void __launch_bounds__(kT, 2) k_spmm(SpParams p, const float *__restrict__ x,
                                             float *__restrict__ y) {
    using G = SpGeo<L>;
    constexpr uint32_t nlo = G::nlo;
    constexpr int K = G::K;
    constexpr int MB = G::maxblk;
    extern __shared__ __align__(16) unsigned char smem[];
    const SpSmem lay(p, MB);
    float *xs = (float *)(smem + lay.xs);
    float *nbuf = (float *)(smem + lay.nb);
    constexpr int NBS = (MB + 1) * kB;  // floats per staging buffer
    float *jh = (float *)(smem + lay.jh);
    float *pc = (float *)(smem + lay.pc);
    uint64_t *pl = (uint64_t *)(smem + lay.pl);
    float *plc = (float *)(smem + lay.plc);
    const int mpc = pad_pa(p.maxpa);
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);  // postfix site j | slot << 8
    float *cc = (float *)(smem + lay.cc);              // J/2 of each cross bond
    uint32_t *rqm = (uint32_t *)(smem + lay.rqm);      // per site: bit k = row bit that flips block k
    int64_t *noff = (int64_t *)(smem + lay.noff);
    int *nn = (int *)(smem + lay.nn);
    __shared__ int sh_npa[kB];
    __shared__ float sh_dpre[kB];
    __shared__ int64_t sh_off[kB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = tid & (kB - 1);  // staging column of this thread
    for (int k = tid; k < p.nb; k += kT) jh[k] = p.jhalf[k];
    // postfix coefficients; padding entries point at the zero row of xs
    for (int k = tid; k < p.npost_pad; k += kT) pc[k] = p.jhalf[p.postid[k]];
    for (int q = tid; q < p.ncross; q += kT) {
        cmeta[q] = (uint32_t)p.cross[4 * q + 1] | ((uint32_t)p.cross[4 * q + 3] << 8);
        cc[q] = p.jhalf[p.cross[4 * q + 2]];
    }

    for (int64_t t = blockIdx.x; t < p.nitems; t += gridDim.x) {
        uint32_t hk[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) hk[k] = __ldg(p.items + t * kB + k);
        const int m = p.nup - __popc(hk[0]);
        const uint32_t l0 = __ldg(p.lo_off + m);
        const int n = (int)(__ldg(p.lo_off + m + 1) - l0);
        const int nm = m > 0 ? (int)(l0 - __ldg(p.lo_off + m - 1)) : 0;
        const int np = m < L ? (int)(__ldg(p.lo_off + m + 2) - __ldg(p.lo_off + m + 1)) : 0;
        __syncthreads();  // previous item done with shared memory
        {
            // x of the kB blocks, transposed: row r, block k at swz(r, k)
            const uint32_t hc = hk[col];
            const int64_t offc = hc != kEmpty ? __ldg(p.hi_off + hc) : 0;
            for (int e = tid; e < n * kB; e += kT) {
                const int rr = e >> 3;
                if (hc != kEmpty) cp_async4(xs + swz(rr, col), x + offc + rr);
                else xs[swz(rr, col)] = 0.f;
            }
            cp_commit();
            if (tid < kB) xs[swz(MB, tid)] = 0.f;
        }
        if (warp < kB) {
            // per-block data: active prefix bonds (precomputed CSR), prefix
            // diagonal, cross neighbour blocks and coefficient vectors
            const int k = warp;
            const uint32_t h = hk[k];
            float dpre = 0.f;
            int cnt = 0;
            if (h != kEmpty) {
                const int64_t c0 = __ldg(p.pcsr_off + h), c1 = __ldg(p.pcsr_off + h + 1);
                cnt = (int)(c1 - c0);
                for (int q = lane; q < pad_pa(cnt); q += 32) {
                    const uint64_t ev = q < cnt ? __ldg(p.pcsr + c0 + q) : 0ull;
                    if (q < cnt) pl[k * p.maxpa + q] = ev;
                    plc[k * mpc + q] = q < cnt ? jh[(uint32_t)(ev & 4095u)] : 0.f;
                }
                for (int q = lane; q < p.npre; q += 32) {
                    const int a = p.pre[3 * q], b = p.pre[3 * q + 1];
                    const float j4 = 0.5f * jh[p.pre[3 * q + 2]];
                    dpre += (((h >> a) ^ (h >> b)) & 1u) ? -j4 : j4;
                }
                for (int c = lane; c < p.ncsite; c += 32) {
                    const int a = p.csite[3 * c];
                    const int hb = (int)((h >> a) & 1u);
                    noff[c * kB + k] = __ldg(p.hi_off + (h ^ (1u << a)));
                    nn[c * kB + k] = hb ? np : nm;
                }
            } else {
                for (int c = lane; c < p.ncsite; c += 32) {
                    noff[c * kB + k] = 0;
                    nn[c * kB + k] = 0;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dpre += __shfl_xor_sync(0xffffffffu, dpre, o);
            if (lane == 0) {
                sh_npa[k] = cnt;
                sh_dpre[k] = dpre + p.jcross;
                sh_off[k] = h != kEmpty ? __ldg(p.hi_off + h) : 0;
            }
        }
        // per cross site: bit k set when a row whose bit j is 1 flips block k
        // (a row whose bit j is 0 flips the other valid blocks)
        for (int c = tid; c < p.ncsite; c += kT) {
            uint32_t m1 = 0;
#pragma unroll
            for (int k = 0; k < kB; ++k)
                if (hk[k] != kEmpty && !((hk[k] >> p.csite[3 * c]) & 1u)) m1 |= 1u << k;
            rqm[c] = m1;
        }
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0; k < kB; ++k) valid |= (hk[k] != kEmpty ? 1u : 0u) << k;
        cp_wait_all();
        __syncthreads();

        float acc[K][kB];
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
            for (int k = 0; k < kB; ++k) acc[r][k] = 0.f;

        // postfix bonds: one target rank per row and bond serves the kB blocks
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT;
            if (i < n) {
                const uint16_t *pt = p.ptab + l0 + i;
                const float *pcb = pc;
#pragma unroll 1
                for (int b0 = 0; b0 < p.npost_pad; b0 += 8, pt += 8 * nlo, pcb += 8) {
                    uint32_t t8[8];
#pragma unroll
                    for (int v = 0; v < 8; ++v) t8[v] = __ldg(pt + v * nlo);
#pragma unroll
                    for (int v = 0; v < 8; ++v)
                        if (t8[v] != (uint32_t)MB) fma8(acc[r], pcb[v], xs, (int)t8[v]);
                }
            }
        }
        // Cross site 0 is staged now, behind the prefix streams.
        auto stage_site = [&](int c, float *dst) {
            const int64_t so = noff[c * kB + col];
            const int sn = nn[c * kB + col];
            for (int e = tid; e < sn * kB; e += kT) cp_async4(dst + swz(e >> 3, col), x + so + (e >> 3));
            cp_commit();
        };
        if (p.ncsite > 0) stage_site(0, nbuf);
        // prefix bonds: per block, coalesced streams from its neighbour blocks.
        // Both rows of a thread load each of kPB neighbours before any use
        // (32 loads in flight per thread; the coefficients wait in shared
        // memory): far neighbour blocks come from DRAM and only memory-level
        // parallelism hides that latency.
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const int npa = sh_npa[k];
            const uint64_t *e = pl + k * p.maxpa;
            const float *cf = plc + k * mpc;
            float a[K];
#pragma unroll
            for (int r = 0; r < K; ++r) a[r] = 0.f;
#pragma unroll 1
            for (int q0 = 0; q0 < npa; q0 += kPB) {
                float v[K][kPB];
#pragma unroll
                for (int w = 0; w < kPB; ++w) {
                    const bool ok = q0 + w < npa;
                    const float *src = x + (ok ? (int64_t)(e[q0 + w] >> 12) : 0);
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        const int i = tid + r * kT;
                        v[r][w] = (ok && i < n) ? __ldg(src + i) : 0.f;
                    }
                }
#pragma unroll
                for (int w = 0; w < kPB; ++w) {
                    const float c = cf[q0 + w];
#pragma unroll
                    for (int r = 0; r < K; ++r) a[r] = fmaf(c, v[r][w], a[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < K; ++r) acc[r][k] += a[r];
        }
        // cross bonds: one prefix site at a time, its kB neighbour blocks
        // staged; site c + 1 is copied while site c is used
        uint32_t lw[K];
#pragma unroll
        for (int r = 0; r < K; ++r) lw[r] = __ldg(p.lo_list + l0 + min(tid + r * kT, n - 1));
#pragma unroll 1
        for (int c = 0; c < p.ncsite; ++c) {
            float *nb = nbuf + (c & 1) * NBS;
            __syncthreads();  // site c - 1 done with the other buffer
            if (c + 1 < p.ncsite) {
                stage_site(c + 1, nbuf + ((c + 1) & 1) * NBS);
                cp_wait_1();
            } else {
                cp_wait_all();
            }
            __syncthreads();  // site c staged
            const int q0 = p.csite[3 * c + 1], q1 = p.csite[3 * c + 2];
            const uint32_t m1 = rqm[c], m0 = valid & ~m1;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const int i = tid + r * kT;
                if (i < n) {
                    const uint32_t l = lw[r];
                    float4 xlo, xhi;
                    row8(xs, i, xlo, xhi);
                    const float xv[kB] = {xlo.x, xlo.y, xlo.z, xlo.w, xhi.x, xhi.y, xhi.z, xhi.w};
#pragma unroll 1
                    for (int q = q0; q < q1; ++q) {
                        const uint32_t meta = cmeta[q];
                        const uint32_t fm = ((l >> (meta & 31u)) & 1u) ? m1 : m0;
                        if (fm) {
                            const uint32_t r2 = __ldg(p.xtab + (meta >> 8) * nlo + (l0 + i));
                            const float cq = cc[q];
                            float4 nlo4, nhi4;
                            row8(nb, (int)r2, nlo4, nhi4);
                            const float nv[kB] = {nlo4.x, nlo4.y, nlo4.z, nlo4.w, nhi4.x, nhi4.y, nhi4.z, nhi4.w};
#pragma unroll
                            for (int k = 0; k < kB; ++k)
                                if ((fm >> k) & 1u) acc[r][k] = fmaf(cq, nv[k] - xv[k], acc[r][k]);
                        }
                    }
                }
            }
        }
        // diagonal and store (coalesced per block)
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT;
            if (i < n) {
                const float dp = __ldg(p.dpost + l0 + i);
#pragma unroll
                for (int k = 0; k < kB; ++k)
                    if (hk[k] != kEmpty) y[sh_off[k] + i] = (sh_dpre[k] + dp) * xs[swz(i, k)] + acc[r][k];
            }
        }
    }
}

// active prefix bonds of every prefix: (row offset of h ^ m_b) << 12 | bond
__global__ void k_pcsr_count(int P, int nup, int L, const int32_t *__restrict__ pre, int npre,
                             int64_t *__restrict__ cnt) {
    const uint64_t nh = 1ull << P;
    for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh;
         h += (uint64_t)gridDim.x * blockDim.x) {
        const int m = nup - __popcll(h);
        int c = 0;
        if (m >= 0 && m <= L)
            for (int q = 0; q < npre; ++q) c += ((h >> pre[3 * q]) ^ (h >> pre[3 * q + 1])) & 1ull;
        cnt[h] = c;
    }
}

__global__ void k_pcsr_fill(int P, int nup, int L, const int32_t *__restrict__ pre, int npre,
                            const int64_t *__restrict__ hi_off, const int64_t *__restrict__ off,
                            uint64_t *__restrict__ out) {
    const uint64_t nh = 1ull << P;
    for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh;
         h += (uint64_t)gridDim.x * blockDim.x) {
        const int m = nup - __popcll(h);
        if (m < 0 || m > L) continue;
        int64_t w = off[h];
        for (int q = 0; q < npre; ++q) {
            const int a = pre[3 * q], b = pre[3 * q + 1];
            if (((h >> a) ^ (h >> b)) & 1ull) {
                const uint64_t h2 = h ^ ((1ull << a) | (1ull << b));
                out[w++] = ((uint64_t)hi_off[h2] << 12) | (uint64_t)pre[3 * q + 2];
            }
        }
    }
}

int spmm_L(int N) { return std::min(12, N - 12); }

}  // namespace

bool spmm_layout_wanted(const xd_basis_s *b) {
    if (b->sym || b->N < 24 || b->nb > 4095) return false;
    const int L = spmm_L(b->N);
    return L >= 10 && b->N - L <= 26;
}

xd_status spmm_layout_build(xd_basis_s *b) {
    SpmmLayoutHost &s = b->spmm;
    const int N = b->N, nup = b->nup;
    const int L = spmm_L(N), P = N - L;
    s.L = L;
    s.P = P;
    // U(1) two-table layout at this L, bond classes and target tables
    U1Layout lay;
    u1_layout_at(N, nup, L, &lay);
    BlockTables T;
    block_tables(N, nup, L, (const int32_t *)b->bonds.data(), b->nb, lay.lo_rank, lay.lo_list, &T, false);
    s.h_lo_off = lay.lo_off;
    s.h_lo_list = lay.lo_list;
    const std::vector<uint32_t> &lo_list = lay.lo_list;
    const std::vector<int64_t> &hi_off = lay.hi_off;
    const std::vector<int32_t> &pre = T.pre, &cross = T.cross, &csite = T.csite;
    const std::vector<uint16_t> &ptab = T.ptab, &xtab = T.xtab;
    s.post.assign(T.post.begin(), T.post.end());
    s.npost = (int)T.post.size();
    s.npost_pad = T.npost_pad;
    s.npre = (int)pre.size() / 3;
    s.ncross = (int)cross.size() / 4;
    s.ncsite = (int)csite.size() / 3;
    s.maxblk = T.maxblk;
    s.h_pre = pre;
    s.h_csite = csite;
    s.cross_ids.clear();
    for (int q = 0; q < s.ncross; ++q) s.cross_ids.push_back(cross[4 * q + 2]);
    std::vector<uint16_t> postid(T.post.begin(), T.post.end());
    postid.resize(s.npost_pad, 0);
    const std::vector<uint32_t> items = prefix_items(P, nup, L, kB, kEmpty);
    s.nitems = (int64_t)items.size() / kB;
    auto up = [](auto **dst, const auto &v) -> xd_status {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        XD_CUDA(dev_malloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(E)));
        if (!v.empty()) XD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
        return XD_OK;
    };
    XD_TRY(up(&s.d_hi_off, hi_off));
    XD_TRY(up(&s.d_lo_off, s.h_lo_off));
    XD_TRY(up(&s.d_lo_list, lo_list));
    XD_TRY(up(&s.d_lo_rank, lay.lo_rank));
    XD_TRY(up(&s.d_items, items));
    XD_TRY(up(&s.d_ptab, ptab));
    XD_TRY(up(&s.d_xtab, xtab));
    XD_TRY(up(&s.d_pre, pre));
    XD_TRY(up(&s.d_cross, cross));
    XD_TRY(up(&s.d_csite, csite));
    XD_TRY(up(&s.d_postid, postid));
    // per-prefix lists of active prefix bonds, built on the device
    {
        const uint64_t nh = 1ull << P;
        int64_t *cnt = nullptr;
        XD_CUDA(dev_malloc((void **)&cnt, (nh + 1) * sizeof(int64_t)));
        const int grid = grid_for((int64_t)nh, 256, 16);
        k_pcsr_count<<<grid, 256>>>(P, nup, L, s.d_pre, s.npre, cnt);
        std::vector<int64_t> hc(nh + 1, 0);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cnt, nh * sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaFree(cnt);
            return cuda_status(e, "prefix list count");
        }
        int64_t run = 0, mx = 0;
        for (uint64_t h = 0; h < nh; ++h) {
            const int64_t c = hc[h];
            hc[h] = run;
            run += c;
            mx = std::max(mx, c);
        }
        hc[nh] = run;
        s.maxpa = (int)std::max<int64_t>(1, mx);
        e = cudaMemcpy(cnt, hc.data(), (nh + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = dev_malloc((void **)&s.d_pcsr, std::max<int64_t>(1, run) * sizeof(uint64_t));
        if (e == cudaSuccess) {
            k_pcsr_fill<<<grid, 256>>>(P, nup, L, s.d_pre, s.npre, s.d_hi_off, cnt, s.d_pcsr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        s.d_pcsr_off = cnt;
        if (e != cudaSuccess) return cuda_status(e, "prefix list fill");
    }
    s.ok = true;
    return XD_OK;
}

void spmm_layout_free(xd_basis_s *b) {
    SpmmLayoutHost &s = b->spmm;
    cudaFree(s.d_hi_off);
    cudaFree(s.d_lo_off);
    cudaFree(s.d_lo_list);
    cudaFree(s.d_lo_rank);
    cudaFree(s.d_items);
    cudaFree(s.d_ptab);
    cudaFree(s.d_xtab);
    cudaFree(s.d_pre);
    cudaFree(s.d_cross);
    cudaFree(s.d_csite);
    cudaFree(s.d_postid);
    cudaFree(s.d_pcsr);
    cudaFree(s.d_pcsr_off);
    s = SpmmLayoutHost();
}

// Per-Hamiltonian tables: J/2 as float and the postfix diagonal per class
// position, d_post(l) = sum over postfix bonds of J/4 (+1 equal, -1 opposite).
xd_status spmm_ham_tables(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    const uint32_t nlo = 1u << s.L;
    std::vector<float> dpost(nlo), jhalf(b->nb);
    for (int k = 0; k < b->nb; ++k) jhalf[k] = (float)(0.5 * h->J[k]);
    for (uint32_t g = 0; g < nlo; ++g) {
        const uint32_t l = s.h_lo_list[g];
        double d = 0.0;
        for (int k : s.post) {
            const int i = b->bonds[k].i, j = b->bonds[k].j;
            d += (((l >> i) & 1) == ((l >> j) & 1) ? 0.25 : -0.25) * h->J[k];
        }
        dpost[g] = (float)d;
    }
    if (!h->d_sp_dpost) XD_CUDA(dev_malloc((void **)&h->d_sp_dpost, nlo * sizeof(float)));
    if (!h->d_sp_jhalf) XD_CUDA(dev_malloc((void **)&h->d_sp_jhalf, std::max(1, b->nb) * sizeof(float)));
    XD_CUDA(cudaMemcpy(h->d_sp_dpost, dpost.data(), nlo * sizeof(float), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_sp_jhalf, jhalf.data(), b->nb * sizeof(float), cudaMemcpyHostToDevice));
    double q = 0.0;
    for (int k : s.cross_ids) q += h->J[k];
    h->sp_jcross = (float)(0.25 * q);
    return XD_OK;
}

template <int L>
static xd_status launch_spmm(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    SpParams p;
    p.nup = b->nup;
    p.hi_off = s.d_hi_off;
    p.lo_off = s.d_lo_off;
    p.lo_list = s.d_lo_list;
    p.items = s.d_items;
    p.nitems = s.nitems;
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
    const SpSmem lay(p, SpGeo<L>::maxblk);
    auto kern = k_spmm<L>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, lay.total));
    if (per_sm < 1) {
        set_error("batched product: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    grid_for(1, 1, 1);
    const int grid = (int)std::min<int64_t>(s.nitems, (int64_t)g_num_sms * per_sm);
    kern<<<grid, kT, lay.total, st>>>(p, (const float *)x, (float *)y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status spmm_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    switch (h->b->spmm.L) {
        case 10: return launch_spmm<10>(h, x, y, st);
        case 11: return launch_spmm<11>(h, x, y, st);
        case 12: return launch_spmm<12>(h, x, y, st);
        default: return launch_spmm<13>(h, x, y, st);
    }
}

}  // namespace xd

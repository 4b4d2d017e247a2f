// xd_u1_block.cu -- block-structured y = H x on large U(1) blocks.
//
// Same product as xd_u1.cu (Eq. 1, pull form), organised around the
// prefix/postfix split of the index layout.  XDiag distributes states by
// prefix and applies postfix-only terms locally (Sec. 5.3); here one CTA
// owns one prefix block h (the C(L, m) consecutive rows sharing the prefix,
// m = nup - popcount(h)) and the bonds fall into three kinds:
//   postfix bonds (both sites < L): the flipped state stays in block h; its
//       rank inside the block comes from a per-postfix-state neighbour list
//       (CSR of (rank, bond) for every L-bit word) and x of the whole block
//       is staged in shared memory, so these gathers are shared-memory loads;
//   prefix bonds (both sites >= L): the flip maps block h to block h ^ m_b
//       with the same in-block rank, so row i reads x[off(h') + i]: one
//       coalesced stream per active bond, decided once per block;
//   cross bonds (one site each side): the flip changes the prefix bit (one
//       neighbour block per bond, decided once per block) and one postfix
//       bit of l; the in-class rank of the new postfix word comes from two
//       small shared tables (high part offsets, low part ranks).
// The diagonal is d_pre(h) + d_post(l) + the cross-bond terms.  Blocks are
// processed largest first (static round robin over the size-sorted list).

#include <algorithm>
#include <vector>

#include "xd_internal.cuh"

namespace xd {

namespace {

struct PreEnt {
    int64_t off;
    double coef;
};
struct CrossEnt {
    int64_t off;   // first row of the neighbour block
    double coef;   // J/2
    int j;         // postfix site
    int req;       // value of bit j that makes the bond flip
    int mcls;      // class (postfix popcount) of the flipped postfix word
    int pad;
};

struct BlkParams {
    U1View u;
    const uint32_t *order;
    int64_t nblk;
    const uint32_t *csr_off;
    const uint32_t *csr;
    const uint16_t *off2;  // [(L+1)][2^(L-w)]
    const uint8_t *rank8;  // [2^w]
    int w;
    const double *dpost;   // [2^L]
    const double *J;       // [nb]
    const int32_t *pre;    // [npre][3]: prefix bit a, prefix bit b, bond id
    int npre;
    const int32_t *cross;  // [ncross][3]: prefix bit, postfix site, bond id
    int ncross;
    int nb;
    int maxblk;
};

template <typename T>
struct SmemLayout {
    size_t xs, off2, rank8, coef, pre, cross, total;
    __host__ __device__ SmemLayout(const BlkParams &p) {
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;
        o += (size_t)p.maxblk * sizeof(T);
        al(16);
        off2 = o;
        o += (size_t)(p.u.L + 1) * (1u << (p.u.L - p.w)) * sizeof(uint16_t);
        al(16);
        rank8 = o;
        o += (size_t)(1u << p.w);
        al(16);
        coef = o;
        o += (size_t)p.nb * sizeof(T);
        al(16);
        pre = o;
        o += (size_t)p.npre * sizeof(PreEnt);
        al(16);
        cross = o;
        o += (size_t)p.ncross * sizeof(CrossEnt);
        al(16);
        total = o;
    }
};

template <typename T>
__global__ void __launch_bounds__(256) k_block_apply(BlkParams p, const T *__restrict__ x,
                                                     T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout<T> lay(p);
    T *xs = (T *)(smem + lay.xs);
    uint16_t *off2 = (uint16_t *)(smem + lay.off2);
    uint8_t *rank8 = (uint8_t *)(smem + lay.rank8);
    T *coef = (T *)(smem + lay.coef);
    PreEnt *pl = (PreEnt *)(smem + lay.pre);
    CrossEnt *cl = (CrossEnt *)(smem + lay.cross);
    __shared__ int sh_npa;
    __shared__ double sh_dpre;

    const U1View &u = p.u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hw = u.L - p.w;
    for (int k = tid; k < (u.L + 1) << hw; k += blockDim.x) off2[k] = p.off2[k];
    for (int k = tid; k < (1 << p.w); k += blockDim.x) rank8[k] = p.rank8[k];
    for (int k = tid; k < p.nb; k += blockDim.x) coef[k] = (T)(0.5 * p.J[k]);
    const uint32_t wmask = (1u << p.w) - 1;

    for (int64_t t = blockIdx.x; t < p.nblk; t += gridDim.x) {
        const uint64_t h = p.order[t];
        const int m = u.nup - __popcll(h);
        const uint32_t l0 = __ldg(u.lo_off + m);
        const int n = (int)(__ldg(u.lo_off + m + 1) - l0);
        const int64_t off = __ldg(u.hi_off + h);
        __syncthreads();  // previous block done with shared memory
        for (int i = tid; i < n; i += blockDim.x) xs[i] = x[off + i];
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
                    pl[pos].off = __ldg(u.hi_off + (h ^ ((1ull << a) | (1ull << b))));
                    pl[pos].coef = 0.5 * Jq;
                }
                cnt += __popc(bal);
            }
            for (int q = lane; q < p.ncross; q += 32) {
                const int a = p.cross[3 * q], j = p.cross[3 * q + 1];
                const double Jq = p.J[p.cross[3 * q + 2]];
                const int hb = (int)((h >> a) & 1);
                CrossEnt e;
                e.off = __ldg(u.hi_off + (h ^ (1ull << a)));
                e.coef = 0.5 * Jq;
                e.j = j;
                e.req = 1 - hb;
                e.mcls = hb ? m + 1 : m - 1;
                e.pad = 0;
                cl[q] = e;
                dpre += 0.25 * Jq;  // cross bonds start at +J/4; flips subtract J/2
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dpre += __shfl_xor_sync(0xffffffffu, dpre, o);
            if (lane == 0) {
                sh_npa = cnt;
                sh_dpre = dpre;
            }
        }
        __syncthreads();
        const int npa = sh_npa;
        const T dpre = (T)sh_dpre;
        for (int i = tid; i < n; i += blockDim.x) {
            const uint32_t l = __ldg(u.lo_list + l0 + i);
            T acc = T(0), dsub = T(0);
            // postfix bonds: shared-memory gathers inside the block
            const uint32_t e1 = __ldg(p.csr_off + l + 1);
            for (uint32_t e = __ldg(p.csr_off + l); e < e1; ++e) {
                const uint32_t v = __ldg(p.csr + e);
                acc += coef[v >> 16] * xs[v & 0xffffu];
            }
            // prefix bonds: coalesced streams from the neighbour blocks
            for (int q = 0; q < npa; ++q) acc += (T)pl[q].coef * x[pl[q].off + i];
            // cross bonds
            for (int q = 0; q < p.ncross; ++q) {
                const CrossEnt &e = cl[q];
                if ((int)((l >> e.j) & 1) == e.req) {
                    const uint32_t l2 = l ^ (1u << e.j);
                    const int r2 = off2[(e.mcls << hw) + (l2 >> p.w)] + rank8[l2 & wmask];
                    const T c = (T)e.coef;
                    acc += c * x[e.off + r2];
                    dsub += c;
                }
            }
            const T d = dpre + (T)__ldg(p.dpost + l) - dsub;
            y[off + i] = d * xs[i] + acc;
        }
    }
}

}  // namespace

// ------------------------------------------------------------ host side

static int64_t binom_h(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

bool block_layout_wanted(const xd_basis_s *b) { return !b->sym && b->N >= 20 && b->L >= 10; }

xd_status block_layout_build(xd_basis_s *b) {
    const int L = b->L, P = b->P, N = b->N, nup = b->nup;
    BlockLayoutHost &bl = b->blk;
    bl.w = std::min(8, L);
    const int hw = L - bl.w;
    // classify bonds
    std::vector<int32_t> pre, cross;
    std::vector<int> post;
    for (int k = 0; k < b->nb; ++k) {
        int i = b->bonds[k].i, j = b->bonds[k].j;
        if (i > j) std::swap(i, j);
        if (j < L) post.push_back(k);
        else if (i >= L) pre.insert(pre.end(), {i - L, j - L, k});
        else cross.insert(cross.end(), {j - L, i, k});
    }
    bl.npre = (int)pre.size() / 3;
    bl.ncross = (int)cross.size() / 3;
    bl.post = post;
    // CSR of postfix flips for every L-bit word: (rank of the flipped word
    // inside its popcount class, bond id)
    const uint32_t nlo = 1u << L;
    std::vector<uint32_t> off(nlo + 1, 0), ent;
    ent.reserve((size_t)nlo * post.size() / 2 + 16);
    for (uint32_t l = 0; l < nlo; ++l) {
        off[l] = (uint32_t)ent.size();
        for (int k : post) {
            int i = b->bonds[k].i, j = b->bonds[k].j;
            if (((l >> i) & 1) == ((l >> j) & 1)) continue;
            uint32_t t = l ^ (1u << i) ^ (1u << j);
            ent.push_back(b->h_lo_rank[t] | ((uint32_t)k << 16));
        }
    }
    off[nlo] = (uint32_t)ent.size();
    // two-level in-class rank tables
    std::vector<uint16_t> off2((size_t)(L + 1) << hw, 0);
    for (int mcls = 0; mcls <= L; ++mcls) {
        uint32_t run = 0;
        for (uint32_t a = 0; a < (1u << hw); ++a) {
            off2[((size_t)mcls << hw) + a] = (uint16_t)run;
            run += (uint32_t)binom_h(bl.w, mcls - __builtin_popcount(a));
        }
    }
    std::vector<uint8_t> rank8(1u << bl.w);
    {
        std::vector<int> cnt(bl.w + 1, 0);
        for (uint32_t v = 0; v < (1u << bl.w); ++v) rank8[v] = (uint8_t)cnt[__builtin_popcount(v)]++;
    }
    // non-empty prefix blocks, largest first
    std::vector<uint32_t> order;
    for (uint64_t h = 0; h < (1ull << P); ++h) {
        int m = nup - __builtin_popcountll(h);
        if (m >= 0 && m <= L) order.push_back((uint32_t)h);
    }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
        return binom_h(L, nup - __builtin_popcount(a)) > binom_h(L, nup - __builtin_popcount(c));
    });
    bl.nblk = (int64_t)order.size();
    bl.maxblk = (int)binom_h(L, L / 2);
    (void)N;
    auto up = [](auto **dst, const auto &v) -> xd_status {
        using E = typename std::remove_reference<decltype(v)>::type::value_type;
        XD_CUDA(cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(E)));
        if (!v.empty()) XD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
        return XD_OK;
    };
    XD_TRY(up(&bl.d_order, order));
    XD_TRY(up(&bl.d_csr_off, off));
    XD_TRY(up(&bl.d_csr, ent));
    XD_TRY(up(&bl.d_off2, off2));
    XD_TRY(up(&bl.d_rank8, rank8));
    XD_TRY(up(&bl.d_pre, pre));
    XD_TRY(up(&bl.d_cross, cross));
    bl.ok = true;
    return XD_OK;
}

void block_layout_free(xd_basis_s *b) {
    BlockLayoutHost &bl = b->blk;
    cudaFree(bl.d_order);
    cudaFree(bl.d_csr_off);
    cudaFree(bl.d_csr);
    cudaFree(bl.d_off2);
    cudaFree(bl.d_rank8);
    cudaFree(bl.d_pre);
    cudaFree(bl.d_cross);
    bl = BlockLayoutHost();
}

// d_post(l) = sum over postfix bonds of J/4 (+1 equal spins, -1 opposite)
xd_status block_ham_tables(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const uint32_t nlo = 1u << b->L;
    std::vector<double> dpost(nlo, 0.0);
    for (uint32_t l = 0; l < nlo; ++l) {
        double d = 0.0;
        for (int k : b->blk.post) {
            int i = b->bonds[k].i, j = b->bonds[k].j;
            d += (((l >> i) & 1) == ((l >> j) & 1) ? 0.25 : -0.25) * h->J[k];
        }
        dpost[l] = d;
    }
    if (!h->d_dpost) XD_CUDA(cudaMalloc((void **)&h->d_dpost, nlo * sizeof(double)));
    XD_CUDA(cudaMemcpy(h->d_dpost, dpost.data(), nlo * sizeof(double), cudaMemcpyHostToDevice));
    return XD_OK;
}

template <typename T>
static xd_status launch_block(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const BlockLayoutHost &bl = b->blk;
    BlkParams p;
    p.u = b->u1view();
    p.order = bl.d_order;
    p.nblk = bl.nblk;
    p.csr_off = bl.d_csr_off;
    p.csr = bl.d_csr;
    p.off2 = bl.d_off2;
    p.rank8 = bl.d_rank8;
    p.w = bl.w;
    p.dpost = h->d_dpost;
    p.J = h->d_J;
    p.pre = bl.d_pre;
    p.npre = bl.npre;
    p.cross = bl.d_cross;
    p.ncross = bl.ncross;
    p.nb = b->nb;
    p.maxblk = bl.maxblk;
    const SmemLayout<T> lay(p);
    auto kern = k_block_apply<T>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, lay.total));
    if (per_sm < 1) {
        set_error("block kernel: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    grid_for(1, 1, 1);
    const int grid = (int)std::min<int64_t>(bl.nblk, (int64_t)g_num_sms * per_sm);
    kern<<<grid, 256, lay.total, st>>>(p, (const T *)x, (T *)y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status block_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt, cudaStream_t st) {
    if (dt == XD_F64) return launch_block<double>(h, x, y, st);
    return launch_block<float>(h, x, y, st);
}

}  // namespace xd

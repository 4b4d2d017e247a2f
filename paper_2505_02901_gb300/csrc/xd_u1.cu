// xd_u1.cu -- y = H x and per-bond bilinear forms on U(1) blocks.
//
// Pull form (the "apply" of Sec. 3.5 with the vector fill of Sec. 5.1):
// every row r of y is written once, no atomics.  For row r with state s
// (a1: unranked from the two-table layout, Sec. 5.2) and every bond b:
//   a2  equal spins:     +J_b/4 x_r on the diagonal
//   a3  opposite spins:  -J_b/4 x_r and +J_b/2 x_c, c = index(s ^ m_b)
//   a4  c from the prefix/postfix tables: c = hi_off[s'>>L] + lo_rank[s'&mask]
//   a5  gather x_c and accumulate.
// The diagonal is written as J_sum/4 - sum over flipped bonds of J_b/2.

#include <algorithm>
#include <mutex>

#include "xd_internal.cuh"
#include "xd_u1_rows.cuh"

namespace xd {

namespace {

constexpr int kThreads = 256;

using namespace u1rows;

// y = H x (the row loop of xd_u1_rows.cuh).
template <typename T, int NV>
__global__ void __launch_bounds__(kThreads) k_apply(U1View u, const double *__restrict__ bond,
                                                    int nb, const T *__restrict__ x,
                                                    T *__restrict__ y) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sm_mask = (uint64_t *)smem;
    T *sm_half = (T *)(sm_mask + nb);
    __shared__ uint64_t sh_range[2];
    stage_bonds(bond, nb, sm_mask, sm_half);
    const T jq = (T)bond[2 * nb];
    __syncthreads();
    apply_rows<T, NV, false>(u, sm_mask, sm_half, nb, jq, x, y, sh_range);
}

// State words of rows [first, first + count): the block of row r is the last
// h with hi_off[h] <= r (binary search), its word (h << L) | lo_list[...].
__global__ void k_states_range(U1View u, int64_t first, int64_t count, uint64_t *__restrict__ out) {
    const uint64_t nh = 1ull << u.P;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = first + q;
        const uint64_t h = find_block(u.hi_off, 0, nh - 1, r);
        const int m = u.nup - __popcll(h);
        const uint32_t l = __ldg(u.lo_list + __ldg(u.lo_off + m) + (uint32_t)(r - __ldg(u.hi_off + h)));
        out[q] = (h << u.L) | l;
    }
}

// Bonds per launch of the bilinear kernel.
constexpr int kChunk = 256;

// Per-bond bilinear forms: part[cta][b] = sum over the CTA's rows of
// g_r (S_i.S_j x)_r (Sec. 3.7 inner, per bond).  With p_r = g_r x_r and
// P = sum_r p_r,
//   <g|S_i.S_j|x> = 1/4 sum_r eps_b(s_r) p_r + 1/2 sum_{r: b flips} g_r x_c
//                 = 1/4 (P - 2 F'_b) + 1/2 F_b,
// F'_b = sum over flipping rows of p_r and F_b = sum over them of g_r x_c
// (eps = +1 for parallel, -1 for antiparallel spins): only the flipping
// bonds of a row cost arithmetic.  A CTA stages the states, g and p of a
// tile of kBT rows in shared memory; warp w owns bonds w, w + 32, ... of the
// chunk and every lane walks a fixed set of the tile's rows, so all sums run
// in a fixed order (lane partials, a fixed shuffle tree, then the CTA
// partial of each bond).  MBW = most bonds per warp.
constexpr int kBT = 1024;
template <typename T, int MBW, bool ZZ>
__global__ void __launch_bounds__(kBT) k_bilinear_bp(U1View u, const uint64_t *__restrict__ masks,
                                                     int nb, int b0, const T *__restrict__ g,
                                                     const T *__restrict__ x,
                                                     double *__restrict__ part, int nv) {
    // nv > 1: column of row-major [dim][nv] vectors (g, x point at the column)
    __shared__ uint64_t sh_s[kBT];
    __shared__ double sh_g[kBT], sh_p[kBT];
    __shared__ double sh_red[kBT / 32];
    __shared__ uint64_t sh_range[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nbc = min(kChunk, nb - b0);
    uint64_t mk[MBW];
    double F[MBW], Fd[MBW];
#pragma unroll
    for (int j = 0; j < MBW; ++j) {
        const int b = warp + 32 * j;
        mk[j] = b < nbc ? __ldg(masks + b0 + b) : 0ull;
        F[j] = 0.0;
        Fd[j] = 0.0;
    }
    double P = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * kBT; base < u.dim; base += (int64_t)gridDim.x * kBT) {
        const int64_t r = base + tid;
        const RowState rs = unrank_tile(u, base, r, sh_range);
        const double gr = rs.valid ? (double)g[r * nv] : 0.0;
        const double pr = rs.valid ? gr * (double)x[r * nv] : 0.0;
        P += pr;
        sh_s[tid] = rs.s;
        sh_g[tid] = gr;
        sh_p[tid] = pr;
        __syncthreads();
        const int nrows = (int)min((int64_t)kBT, u.dim - base);
#pragma unroll 2
        for (int rr = lane; rr < nrows; rr += 32) {
            const uint64_t s = sh_s[rr];
            const double gq = sh_g[rr], pq = sh_p[rr];
#pragma unroll
            for (int j = 0; j < MBW; ++j) {
                const uint64_t tb = s & mk[j];
                if (tb != 0 && tb != mk[j]) {
                    if (!ZZ) {
                        const int64_t c = rank_of(u, s ^ mk[j]);
                        F[j] = fma(gq, (double)__ldg(x + c * nv), F[j]);
                    }
                    Fd[j] += pq;
                }
            }
        }
        // the next tile overwrites the staged rows after unrank_tile's barrier
    }
#pragma unroll
    for (int j = 0; j < MBW; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            F[j] += __shfl_xor_sync(0xffffffffu, F[j], o);
            Fd[j] += __shfl_xor_sync(0xffffffffu, Fd[j], o);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) P += __shfl_xor_sync(0xffffffffu, P, o);
    if (lane == 0) sh_red[warp] = P;
    __syncthreads();
    double Pb = 0.0;
    for (int w = 0; w < kBT / 32; ++w) Pb += sh_red[w];
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < MBW; ++j) {
            const int b = warp + 32 * j;
            if (b < nbc) part[(size_t)blockIdx.x * nb + b0 + b] = 0.25 * (Pb - 2.0 * Fd[j]) + (ZZ ? 0.0 : 0.5 * F[j]);
        }
}

// out[b] = sum_c part[c][b] in fixed order.
__global__ void k_sum_columns(const double *__restrict__ part, int rows, int cols,
                              double *__restrict__ out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= cols) return;
    double s = 0.0;
    for (int c = 0; c < rows; ++c) s += part[(size_t)c * cols + b];
    out[b] = s;
}

}  // namespace

template <typename T, int NV>
static xd_status launch_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    const double *bondbuf = h->d_bond;
    const U1View u = h->b->u1view();
    const int nb = h->b->nb;
    size_t smem = (size_t)nb * (sizeof(uint64_t) + sizeof(T));
    auto kern = k_apply<T, NV>;
    if (smem > 48 * 1024) XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = grid_for(u.dim, kThreads, 8);
    kern<<<grid, kThreads, smem, st>>>(u, bondbuf, nb, (const T *)x, (T *)y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status u1_states(const xd_basis_s *b, int64_t first, int64_t count, uint64_t *out, cudaStream_t st) {
    const int grid = grid_for(count, kThreads, 8);
    k_states_range<<<grid, kThreads, 0, st>>>(b->u1view(), first, count, out);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status u1_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt, int nvec,
                   cudaStream_t st) {
    if (nvec == 1 && dt == XD_F32 && h->b->spmm.ok) return spmm_apply(h, x, y, st);
    if (nvec == 1 && dt == XD_F64 && passes_usable(h)) {
        const xd_status s = passes_apply_f64(h, x, y, st);
        // a workspace that does not fit, or prefix bonds that four windows
        // cannot hold, send this product to the FP64 block kernel
        if (s != XD_ENOMEM && s != XD_ERANGE) return s;
    }
    if (nvec == 8 && dt == XD_F32 && spmm8_usable(h, x, y)) return spmm8_apply(h, x, y, st);
    if (nvec == 1 && h->b->blk.ok) return block_apply(h, x, y, dt, st);
    if (dt == XD_F64) {
        switch (nvec) {
            case 1: return launch_apply<double, 1>(h, x, y, st);
            case 2: return launch_apply<double, 2>(h, x, y, st);
            case 4: return launch_apply<double, 4>(h, x, y, st);
            default: return launch_apply<double, 8>(h, x, y, st);
        }
    }
    switch (nvec) {
        case 1: return launch_apply<float, 1>(h, x, y, st);
        case 2: return launch_apply<float, 2>(h, x, y, st);
        case 4: return launch_apply<float, 4>(h, x, y, st);
        default: return launch_apply<float, 8>(h, x, y, st);
    }
}

template <typename T, bool ZZ = false>
static xd_status launch_bilinear_bp(const U1View &u, const uint64_t *masks, int nb, int grid, const void *g,
                                    const void *x, double *part, cudaStream_t st, int nv = 1) {
    for (int b0 = 0; b0 < nb; b0 += kChunk) {
        const int nbc = std::min(kChunk, nb - b0);
        const int mbw = (nbc + 31) / 32;
        auto go = [&](auto kern) {
            kern<<<grid, kBT, 0, st>>>(u, masks, nb, b0, (const T *)g, (const T *)x, part, nv);
        };
        if (mbw <= 1) go(k_bilinear_bp<T, 1, ZZ>);
        else if (mbw <= 2) go(k_bilinear_bp<T, 2, ZZ>);
        else if (mbw <= 4) go(k_bilinear_bp<T, 4, ZZ>);
        else go(k_bilinear_bp<T, 8, ZZ>);
        XD_CUDA(cudaGetLastError());
    }
    return XD_OK;
}

// dJ[b] = sum over the nv columns of the per-bond forms: the partials of
// column k fill rows [k grid, (k + 1) grid) and one fixed-order sum over all
// rows follows (deterministic).
xd_status u1_bilinear_nvec(const xd_ham_s *h, const void *g, const void *x, xd_dtype dt, int nv, double *dJ,
                           cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const int nb = b->nb;
    const U1View u = b->u1view();
    const int grid = grid_for(u.dim, kBT, 1);
    xd_ham_s *hm = const_cast<xd_ham_s *>(h);
    XD_TRY(ensure_partials(hm, sizeof(double) * (size_t)grid * nb * nv));
    const uint64_t *d_masks = (const uint64_t *)(h->d_bond + nb);
    const size_t es = dt == XD_F64 ? sizeof(double) : sizeof(float);
    for (int k = 0; k < nv; ++k) {
        const void *gk = (const char *)g + k * es, *xk = (const char *)x + k * es;
        double *pk = hm->d_part + (size_t)k * grid * nb;
        if (dt == XD_F64) XD_TRY(launch_bilinear_bp<double>(u, d_masks, nb, grid, gk, xk, pk, st, nv));
        else XD_TRY(launch_bilinear_bp<float>(u, d_masks, nb, grid, gk, xk, pk, st, nv));
    }
    k_sum_columns<<<(nb + 127) / 128, 128, 0, st>>>(hm->d_part, grid * nv, nb, dJ);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

xd_status u1_bilinear(const xd_ham_s *h, const void *g, const void *x, xd_dtype dt, double *dJ,
                      cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const int nb = b->nb;
    const U1View u = b->u1view();
    const int grid = grid_for(u.dim, kBT, 1);
    xd_ham_s *hm = const_cast<xd_ham_s *>(h);
    XD_TRY(ensure_partials(hm, sizeof(double) * (size_t)grid * nb));
    const uint64_t *d_masks = (const uint64_t *)(h->d_bond + nb);
    double *d_part = hm->d_part;
    if (dt == XD_F64) XD_TRY(launch_bilinear_bp<double>(u, d_masks, nb, grid, g, x, d_part, st));
    else XD_TRY(launch_bilinear_bp<float>(u, d_masks, nb, grid, g, x, d_part, st));
    k_sum_columns<<<(nb + 127) / 128, 128, 0, st>>>(d_part, grid, nb, dJ);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free variant of the per-bond bilinear forms.
//
// Some callers cannot let a library call cudaMalloc: a process whose own
// allocator owns all device memory (a pool sized once at start-up, or a hard
// memory budget), or a latency-sensitive loop where cudaMalloc/cudaFree may
// synchronise the device.  xd_apply_bilinear keeps its per-CTA partial sums
// in a workspace that the handle allocates (and grows) on demand; this
// variant keeps them in the fixed file-scope array below instead, so the
// call itself allocates nothing.  Every call, on every stream, shares this
// one array and leaves the last call's partials in it; nothing in it needs
// to start at zero (each launch writes every partial it later reads), but
// two calls that overlap on the GPU race on it and give wrong results.

namespace {

// [kNoAllocCtas][kNoAllocBonds] partial sums: 608 x 256 doubles = 1.19 MiB,
// held on every GPU that loads the library until the process exits.
constexpr int kNoAllocCtas = 608;
constexpr int kNoAllocBonds = 256;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocCtas * kNoAllocBonds];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the name
// g_noalloc_partials is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
xd_status noalloc_scratch(double **out) {
    int dev = 0;
    XD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("xd_apply_bilinear_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
        return XD_ERANGE;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_noalloc_partials)");
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return XD_OK;
}

}  // namespace

}  // namespace xd

extern "C" xd_status xd_apply_bilinear_noalloc(xd_ham h, const void *g, const void *x, xd_dtype dt,
                                               double *dJ, xd_stream stream) {
    using namespace xd;
    if (!h || !g || !x || !dJ) {
        set_error("xd_apply_bilinear_noalloc: NULL argument");
        return XD_EINVAL;
    }
    const xd_basis_s *b = h->b;
    if (b->sym) {
        set_error("xd_apply_bilinear_noalloc: U(1) blocks only (this block is symmetry-adapted)");
        return XD_EINVAL;
    }
    if (dt != XD_F64 && dt != XD_F32) {
        set_error("xd_apply_bilinear_noalloc: dtype must be XD_F64 or XD_F32");
        return XD_EINVAL;
    }
    const int nb = b->nb;
    if (nb > kNoAllocBonds) {
        set_error("xd_apply_bilinear_noalloc: %d bonds exceed the fixed scratch limit of %d bonds "
                  "(use xd_apply_bilinear)", nb, kNoAllocBonds);
        return XD_ERANGE;
    }
    if (b->dim == 0) return XD_OK;
    double *part = nullptr;
    XD_TRY(noalloc_scratch(&part));
    const U1View u = b->u1view();
    const int grid = std::min(grid_for(u.dim, kBT, 1), kNoAllocCtas);
    const uint64_t *masks = (const uint64_t *)(h->d_bond + nb);
    cudaStream_t st = (cudaStream_t)stream;
    if (dt == XD_F64) XD_TRY(launch_bilinear_bp<double>(u, masks, nb, grid, g, x, part, st));
    else XD_TRY(launch_bilinear_bp<float>(u, masks, nb, grid, g, x, part, st));
    k_sum_columns<<<(nb + 127) / 128, 128, 0, st>>>(part, grid, nb, dJ);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// Two-point spin correlations out[p] = <psi| O_{i_p j_p} |psi> on a U(1)
// block: the bilinear kernel with g = x = psi and the pair masks as bonds
// (S_i.S_j), or its diagonal part alone (Sz_i Sz_j, no gathers).  A pair
// with i = j has a one-bit mask that never flips: the kernel returns
// <psi|psi>/4, which is (Sz_i)^2; S_i.S_i = 3/4 is three times that.
extern "C" xd_status xd_correlations(xd_basis b, const void *psi, xd_dtype dt, const int32_t *pairs,
                                     int npairs, int kind, double *out) {
    using namespace xd;
    if (!b || !psi || !out || (npairs > 0 && !pairs)) {
        set_error("xd_correlations: NULL argument");
        return XD_EINVAL;
    }
    if (b->sym ? dt != (b->cplx ? XD_C128 : XD_F64) : (dt != XD_F64 && dt != XD_F32)) {
        set_error(b->sym ? "xd_correlations: a symmetric block takes XD_F64 (real) or XD_C128 (complex)"
                         : "xd_correlations: dtype must be XD_F64 or XD_F32");
        return XD_EINVAL;
    }
    if (kind != 0 && kind != 1) {
        set_error("xd_correlations: kind must be 0 (Sz Sz) or 1 (S.S)");
        return XD_EINVAL;
    }
    if (npairs < 0 || npairs > (1 << 20)) {
        set_error("xd_correlations: npairs = %d out of range", npairs);
        return XD_ERANGE;
    }
    std::vector<uint64_t> m(npairs);
    for (int q = 0; q < npairs; ++q) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        if (i < 0 || i >= b->N || j < 0 || j >= b->N) {
            set_error("xd_correlations: pair %d = (%d, %d) outside 0..%d", q, i, j, b->N - 1);
            return XD_EINVAL;
        }
        m[q] = (1ull << i) | (1ull << j);
    }
    if (npairs == 0) return XD_OK;
    if (b->dim == 0) {
        for (int q = 0; q < npairs; ++q) out[q] = 0.0;
        return XD_OK;
    }
    if (b->sym) return sym_correlations(b, psi, dt, pairs, npairs, kind, out);
    const U1View u = b->u1view();
    const int grid = grid_for(u.dim, kBT, 1);
    uint64_t *d_m = nullptr;
    double *d_part = nullptr, *d_out = nullptr;
    cudaError_t e = dev_malloc((void **)&d_m, sizeof(uint64_t) * npairs);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_part, sizeof(double) * (size_t)grid * npairs);
    if (e == cudaSuccess) e = dev_malloc((void **)&d_out, sizeof(double) * npairs);
    if (e == cudaSuccess) e = cudaMemcpy(d_m, m.data(), sizeof(uint64_t) * npairs, cudaMemcpyHostToDevice);
    xd_status s = e == cudaSuccess ? XD_OK : cuda_status(e, "xd_correlations workspace");
    if (s == XD_OK) {
        if (dt == XD_F64)
            s = kind ? launch_bilinear_bp<double, false>(u, d_m, npairs, grid, psi, psi, d_part, 0)
                     : launch_bilinear_bp<double, true>(u, d_m, npairs, grid, psi, psi, d_part, 0);
        else
            s = kind ? launch_bilinear_bp<float, false>(u, d_m, npairs, grid, psi, psi, d_part, 0)
                     : launch_bilinear_bp<float, true>(u, d_m, npairs, grid, psi, psi, d_part, 0);
    }
    if (s == XD_OK) {
        k_sum_columns<<<(npairs + 127) / 128, 128>>>(d_part, grid, npairs, d_out);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(double) * npairs, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_status(e, "xd_correlations");
    }
    cudaFree(d_m);
    cudaFree(d_part);
    cudaFree(d_out);
    if (s != XD_OK) return s;
    if (kind)
        for (int q = 0; q < npairs; ++q)
            if (pairs[2 * q] == pairs[2 * q + 1]) out[q] *= 3.0;
    return XD_OK;
}

namespace xd {
}  // namespace xd

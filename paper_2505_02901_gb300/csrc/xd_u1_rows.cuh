// xd_u1_rows.cuh -- the row loop of the plain U(1) product (pull form, one
// write per row, no atomics; Sec. 3.5 apply, Sec. 5.2 two-table index) as
// device functions, shared by k_apply (xd_u1.cu) and the persistent Lanczos
// kernel (xd_lanczos.cu).  For row r with state s and every bond b: equal
// spins add +J_b/4 x_r, opposite spins -J_b/4 x_r and +J_b/2 x_c with
// c = index(s ^ m_b); the diagonal is J_sum/4 - sum over flipped bonds J_b/2.

#pragma once

#include "xd_internal.cuh"

namespace xd {

// a product and a fused multiply-add with their roundings fixed (no
// contraction left to the compiler), for arithmetic that two kernels must
// reproduce bit for bit
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

namespace u1rows {

// largest h in [lo, hi] with hi_off[h] <= r (hi_off is non-decreasing)
__device__ __forceinline__ uint64_t find_block(const int64_t *__restrict__ hi_off, uint64_t lo,
                                               uint64_t hi, int64_t r) {
    while (lo < hi) {
        uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(hi_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Row r -> (state, block).  The CTA first brackets the blocks of its rows.
struct RowState {
    uint64_t s;
    bool valid;
};

__device__ __forceinline__ RowState unrank_tile(const U1View &u, int64_t base, int64_t r,
                                                uint64_t *sh_range) {
    // sh_range[0..1]: block range of rows [base, base + blockDim.x)
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t nh = 1ull << u.P;
        int64_t last = min(base + (int64_t)blockDim.x, u.dim) - 1;
        uint64_t h0 = find_block(u.hi_off, 0, nh - 1, base);
        uint64_t h1 = find_block(u.hi_off, h0, nh - 1, last);
        sh_range[0] = h0;
        sh_range[1] = h1;
    }
    __syncthreads();
    RowState rs;
    rs.valid = r < u.dim;
    rs.s = 0;
    if (rs.valid) {
        uint64_t h = find_block(u.hi_off, sh_range[0], sh_range[1], r);
        int64_t i = r - __ldg(u.hi_off + h);
        int m = u.nup - __popcll(h);
        uint32_t l = __ldg(u.lo_list + __ldg(u.lo_off + m) + (uint32_t)i);
        rs.s = (h << u.L) | l;
    }
    return rs;
}

__device__ __forceinline__ int64_t rank_of(const U1View &u, uint64_t t) {
    return __ldg(u.hi_off + (t >> u.L)) + (int64_t)__ldg(u.lo_rank + (t & u.lomask));
}

// x entries: through the read-only path, or (COHERENT) through L2, for a
// vector written earlier by other CTAs of the same kernel
template <typename T, int NV, bool COHERENT>
__device__ __forceinline__ void load_row(const T *x, int64_t c, T (&out)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = COHERENT ? __ldcg(x + c * NV + k) : __ldg(x + c * NV + k);
}

// Bond masks and J_b/2 from the handle's bond table [J (nb) | masks (nb) | sum J / 4].
template <typename T>
__device__ __forceinline__ void stage_bonds(const double *__restrict__ bond, int nb, uint64_t *sm_mask, T *sm_half) {
    const uint64_t *masks = (const uint64_t *)(bond + nb);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        sm_half[b] = (T)(0.5 * bond[b]);
        sm_mask[b] = masks[b];
    }
}

// y = H x on the rows of this CTA (grid-stride tiles of blockDim.x rows);
// every thread of the CTA calls it (the tile unranking has barriers).
template <typename T, int NV, bool COHERENT>
__device__ __forceinline__ void apply_rows(const U1View &u, const uint64_t *sm_mask, const T *sm_half, int nb,
                                           T jq, const T *x, T *y, uint64_t *sh_range) {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < u.dim; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = base + threadIdx.x;
        const RowState rs = unrank_tile(u, base, r, sh_range);
        if (!rs.valid) continue;
        const uint64_t s = rs.s;
        T acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = T(0);
        T dsub = T(0);
        for (int b = 0; b < nb; ++b) {
            const uint64_t mk = sm_mask[b];
            const uint64_t t = s & mk;
            if (t != 0 && t != mk) {
                const int64_t c = rank_of(u, s ^ mk);
                const T cf = sm_half[b];
                T xv[NV];
                load_row<T, NV, COHERENT>(x, c, xv);
#pragma unroll
                for (int k = 0; k < NV; ++k) acc[k] = fma_rn(cf, xv[k], acc[k]);
                dsub += cf;
            }
        }
        T xr[NV];
        load_row<T, NV, COHERENT>(x, r, xr);
        const T d = jq - dsub;
#pragma unroll
        for (int k = 0; k < NV; ++k) y[r * NV + k] = fma_rn(d, xr[k], acc[k]);
    }
}

}  // namespace u1rows
}  // namespace xd

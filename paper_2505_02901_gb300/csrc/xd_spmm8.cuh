// xd_spmm8.cuh -- the FP32 eight-right-hand-side product of one prefix block
// as device functions, shared by the one-operator kernel (xd_u1_spmm8.cu)
// and the batched persistent kernel (xd_batch.cu).  The method is described
// in xd_u1_spmm8.cu.

#pragma once

#include "xd_internal.cuh"

namespace xd {
namespace sp8 {

constexpr int kT8 = 512;      // threads per CTA
constexpr int kPB8 = 2;       // prefix bonds per step (2 rows x 2 bonds x 32 bytes in flight)
constexpr uint32_t kEmpty8 = 0xffffffffu;

template <int L>
struct Sp8Geo {
    static constexpr uint32_t nlo = 1u << L;
    static constexpr int maxblk = L == 12 ? 924 : L == 11 ? 462 : 252;
    static constexpr int K = (maxblk + kT8 - 1) / kT8;  // rows per thread
};

struct Sp8Params {
    int nup;
    const int64_t *hi_off;
    const uint32_t *lo_off, *lo_list;
    const uint32_t *items;      // prefixes (the one-vector layout's items, read one prefix at a time)
    int64_t nprefix;            // entries of items
    const uint16_t *ptab;       // [npost_pad][2^L], "no flip" = maxblk (zero row)
    int npost_pad;
    const uint16_t *xtab;       // [nslot][2^L]
    const float *dpost;         // [2^L] postfix diagonal by class position
    const int64_t *pcsr_off;    // [2^P + 1]
    const uint64_t *pcsr;       // (neighbour block row offset << 12) | bond id
    int maxpa;
    const int32_t *pre;         // [npre][3]
    int npre;
    const int32_t *cross;       // [ncross][4] prefix bit, postfix site, bond id, slot
    int ncross;
    const int32_t *csite;       // [ncsite][3] prefix bit, first, end
    int ncsite;
    const float *jhalf;         // [nb] J/2
    const uint16_t *postid;     // [npost_pad]
    int nb;
    float jcross;
};

__host__ __device__ inline int pad_even(int v) { return (v + kPB8 - 1) / kPB8 * kPB8; }

struct Sp8Smem {
    size_t xs, nb, jh, pc, pl, plc, cmeta, cc, noff, nn, total;
    __host__ __device__ Sp8Smem(const Sp8Params &p, int maxblk) {
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;
        o += (size_t)(maxblk + 1) * 8 * sizeof(float);
        al(128);
        nb = o;  // two staging buffers for cross sites
        o += 2 * (size_t)(maxblk + 1) * 8 * sizeof(float);
        al(16);
        jh = o;
        o += (size_t)p.nb * sizeof(float);
        al(16);
        pc = o;
        o += (size_t)p.npost_pad * sizeof(float);
        al(16);
        pl = o;
        o += (size_t)p.maxpa * sizeof(uint64_t);
        al(16);
        plc = o;
        o += (size_t)pad_even(p.maxpa) * sizeof(float);
        al(16);
        cmeta = o;
        o += (size_t)p.ncross * sizeof(uint32_t);
        al(16);
        cc = o;
        o += (size_t)p.ncross * sizeof(float);
        al(16);
        noff = o;
        o += (size_t)p.ncsite * sizeof(int64_t);
        al(16);
        nn = o;
        o += (size_t)p.ncsite * sizeof(int);
        al(16);
        total = o;
    }
};

__device__ __forceinline__ void cp16(void *smem_dst, const void *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp8_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp8_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp8_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Staged rows are 32 bytes; rows with bit 2 set store their halves swapped
// so that 16-byte loads of consecutive rows hit distinct banks.
__device__ __forceinline__ int half_at(int r, int hf) { return r * 8 + ((hf ^ ((r >> 2) & 1)) << 2); }

__device__ __forceinline__ void row8s(const float *base, int r, float (&v)[8]) {
    const float4 lo = *(const float4 *)(base + half_at(r, 0));
    const float4 hi = *(const float4 *)(base + half_at(r, 1));
    v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
    v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
}

// rows [0, n) of the block at row offset off (32-byte rows) into dst
__device__ __forceinline__ void stage_rows(float *dst, const float *x, int64_t off, int n, int tid) {
    for (int e = tid; e < 2 * n; e += kT8) {
        const int r = e >> 1, hf = e & 1;
        cp16(dst + half_at(r, hf), x + (off + r) * 8 + 4 * hf);
    }
    cp8_commit();
}

// Per-operator shared tables (J/2 by bond, by postfix slot, cross metadata).
template <int L>
__device__ __forceinline__ void tables(const Sp8Params &p, unsigned char *smem) {
    const Sp8Smem lay(p, Sp8Geo<L>::maxblk);
    float *jh = (float *)(smem + lay.jh);
    float *pc = (float *)(smem + lay.pc);
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);  // postfix site j | slot << 8
    float *cc = (float *)(smem + lay.cc);
    const int tid = threadIdx.x;
    for (int k = tid; k < p.nb; k += kT8) jh[k] = p.jhalf[k];
    for (int k = tid; k < p.npost_pad; k += kT8) pc[k] = p.jhalf[p.postid[k]];
    for (int q = tid; q < p.ncross; q += kT8) {
        cmeta[q] = (uint32_t)p.cross[4 * q + 1] | ((uint32_t)p.cross[4 * q + 3] << 8);
        cc[q] = p.jhalf[p.cross[4 * q + 2]];
    }
}

// Y rows of prefix block h (x, y [dim][8]); starts with a barrier, so the
// previous block's use of shared memory is complete.
template <int L>
__device__ __forceinline__ void block(const Sp8Params &p, unsigned char *smem, uint32_t h,
                                      const float *__restrict__ x, float *__restrict__ y) {
    using G = Sp8Geo<L>;
    constexpr uint32_t nlo = G::nlo;
    constexpr int K = G::K;
    constexpr int MB = G::maxblk;
    constexpr int NBS = (MB + 1) * 8;
    const Sp8Smem lay(p, MB);
    float *xs = (float *)(smem + lay.xs);
    float *nbuf = (float *)(smem + lay.nb);
    float *jh = (float *)(smem + lay.jh);
    float *pc = (float *)(smem + lay.pc);
    uint64_t *pl = (uint64_t *)(smem + lay.pl);
    float *plc = (float *)(smem + lay.plc);
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);  // postfix site j | slot << 8
    float *cc = (float *)(smem + lay.cc);
    int64_t *noff = (int64_t *)(smem + lay.noff);
    int *nn = (int *)(smem + lay.nn);
    __shared__ int sh_npa;
    __shared__ float sh_dpre;
    __shared__ int64_t sh_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = p.nup - __popc(h);
    const uint32_t l0 = __ldg(p.lo_off + m);
    const int n = (int)(__ldg(p.lo_off + m + 1) - l0);
    const int nm = m > 0 ? (int)(l0 - __ldg(p.lo_off + m - 1)) : 0;
    const int np = m < L ? (int)(__ldg(p.lo_off + m + 2) - __ldg(p.lo_off + m + 1)) : 0;
    const int64_t off = __ldg(p.hi_off + h);
    __syncthreads();  // previous block done with shared memory
    stage_rows(xs, x, off, n, tid);
    if (tid < 8) xs[MB * 8 + tid] = 0.f;  // zero row for padded postfix targets
    if (warp == 0) {
        // active prefix bonds with their coefficients; prefix diagonal
        const int64_t c0 = __ldg(p.pcsr_off + h);
        const int cnt = (int)(__ldg(p.pcsr_off + h + 1) - c0);
        for (int q = lane; q < pad_even(cnt); q += 32) {
            const uint64_t ev = q < cnt ? __ldg(p.pcsr + c0 + q) : 0ull;
            if (q < cnt) pl[q] = ev;
            plc[q] = q < cnt ? jh[(uint32_t)(ev & 4095u)] : 0.f;
        }
        float dpre = 0.f;
        for (int q = lane; q < p.npre; q += 32) {
            const int a = p.pre[3 * q], b = p.pre[3 * q + 1];
            const float j4 = 0.5f * jh[p.pre[3 * q + 2]];
            dpre += (((h >> a) ^ (h >> b)) & 1u) ? -j4 : j4;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dpre += __shfl_xor_sync(0xffffffffu, dpre, o);
        if (lane == 0) {
            sh_npa = cnt;
            sh_dpre = dpre + p.jcross;
            sh_off = off;
        }
    } else if (warp == 1) {
        for (int c = lane; c < p.ncsite; c += 32) {
            const int a = p.csite[3 * c];
            noff[c] = __ldg(p.hi_off + (h ^ (1u << a)));
            nn[c] = ((h >> a) & 1u) ? np : nm;
        }
    }
    cp8_wait_all();
    __syncthreads();

    float acc[K][8];
#pragma unroll
    for (int r = 0; r < K; ++r)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[r][k] = 0.f;

    // postfix bonds: one target rank per row and bond serves the 8 columns
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int i = tid + r * kT8;
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
                    if (t8[v] != (uint32_t)MB) {
                        float nv[8];
                        row8s(xs, (int)t8[v], nv);
#pragma unroll
                        for (int k = 0; k < 8; ++k) acc[r][k] = fmaf(pcb[v], nv[k], acc[r][k]);
                    }
            }
        }
    }
    // cross site 0 is staged behind the prefix streams
    if (p.ncsite > 0) stage_rows(nbuf, x, noff[0], nn[0], tid);
    // prefix bonds: rows of the neighbour blocks read in place, 32 bytes
    // per row; kPB8 bonds x K rows of loads in flight per thread
    const int npa = sh_npa;
#pragma unroll 1
    for (int q0 = 0; q0 < npa; q0 += kPB8) {
        float4 v[K][kPB8][2];
#pragma unroll
        for (int w = 0; w < kPB8; ++w) {
            const bool ok = q0 + w < npa;
            const float *src = x + (ok ? (int64_t)(pl[q0 + w] >> 12) * 8 : 0);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const int i = tid + r * kT8;
                if (ok && i < n) {
                    v[r][w][0] = __ldg((const float4 *)(src + (int64_t)i * 8));
                    v[r][w][1] = __ldg((const float4 *)(src + (int64_t)i * 8 + 4));
                } else {
                    v[r][w][0] = v[r][w][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
#pragma unroll
        for (int w = 0; w < kPB8; ++w) {
            const float c = plc[q0 + w];
#pragma unroll
            for (int r = 0; r < K; ++r) {
                acc[r][0] = fmaf(c, v[r][w][0].x, acc[r][0]);
                acc[r][1] = fmaf(c, v[r][w][0].y, acc[r][1]);
                acc[r][2] = fmaf(c, v[r][w][0].z, acc[r][2]);
                acc[r][3] = fmaf(c, v[r][w][0].w, acc[r][3]);
                acc[r][4] = fmaf(c, v[r][w][1].x, acc[r][4]);
                acc[r][5] = fmaf(c, v[r][w][1].y, acc[r][5]);
                acc[r][6] = fmaf(c, v[r][w][1].z, acc[r][6]);
                acc[r][7] = fmaf(c, v[r][w][1].w, acc[r][7]);
            }
        }
    }
    // cross bonds: site by site, site c + 1 copied while site c is used;
    // row l flips with bond (a, j) when bit j of l differs from bit a of h
    uint32_t lw[K];
#pragma unroll
    for (int r = 0; r < K; ++r) lw[r] = __ldg(p.lo_list + l0 + min(tid + r * kT8, n - 1));
#pragma unroll 1
    for (int c = 0; c < p.ncsite; ++c) {
        const float *nb = nbuf + (c & 1) * NBS;
        __syncthreads();  // site c - 1 done with the other buffer
        if (c + 1 < p.ncsite) {
            stage_rows(nbuf + ((c + 1) & 1) * NBS, x, noff[c + 1], nn[c + 1], tid);
            cp8_wait_1();
        } else {
            cp8_wait_all();
        }
        __syncthreads();  // site c staged
        const int a = p.csite[3 * c], q0 = p.csite[3 * c + 1], q1 = p.csite[3 * c + 2];
        const uint32_t ha = (h >> a) & 1u;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT8;
            if (i < n) {
                float xv[8];
                row8s(xs, i, xv);
#pragma unroll 1
                for (int q = q0; q < q1; ++q) {
                    const uint32_t meta = cmeta[q];
                    if (((lw[r] >> (meta & 31u)) & 1u) != ha) {
                        const int r2 = (int)__ldg(p.xtab + (meta >> 8) * nlo + (l0 + i));
                        const float cq = cc[q];
                        float nv[8];
                        row8s(nb, r2, nv);
#pragma unroll
                        for (int k = 0; k < 8; ++k) acc[r][k] = fmaf(cq, nv[k] - xv[k], acc[r][k]);
                    }
                }
            }
        }
    }
    // diagonal and store: two 16-byte stores per row
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const int i = tid + r * kT8;
        if (i < n) {
            const float d = sh_dpre + __ldg(p.dpost + l0 + i);
            float xv[8];
            row8s(xs, i, xv);
            float *yo = y + (sh_off + i) * 8;
            *(float4 *)yo = make_float4(fmaf(d, xv[0], acc[r][0]), fmaf(d, xv[1], acc[r][1]),
                                        fmaf(d, xv[2], acc[r][2]), fmaf(d, xv[3], acc[r][3]));
            *(float4 *)(yo + 4) = make_float4(fmaf(d, xv[4], acc[r][4]), fmaf(d, xv[5], acc[r][5]),
                                              fmaf(d, xv[6], acc[r][6]), fmaf(d, xv[7], acc[r][7]));
        }
    }

}

}  // namespace sp8

// Parameters of the eight-vector product of h (its U(1) prefix-block layout).
void sp8_params(const xd_ham_s *h, sp8::Sp8Params *p);

}  // namespace xd

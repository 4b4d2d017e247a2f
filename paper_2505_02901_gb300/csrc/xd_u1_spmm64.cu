// xd_u1_spmm64.cu -- FP64 y = H x on large U(1) blocks without FP64
// arithmetic per matrix element.
//
// The product is the one of xd_u1_spmm.cu (Eq. 1, pull form; the
// prefix/postfix view of Sec. 5.3 with H = H_post + H_pre + H_cross, kB
// same-class prefix blocks per work item, x staged transposed in shared
// memory) with FP64 input and output.  GB300 runs FP64 arithmetic at a small
// fraction of its FP32 and integer rates, so one FP64 operation per matrix
// element would bound the product.  Here each element costs FP32 or integer
// operations and each output row a few FP64 operations, in one of two exact
// or FP64-accurate arithmetics, chosen per Hamiltonian:
//
// Fixed point (couplings that are small integer multiples k_b q of one
// quantum q, e.g. J1 = 1, J2 = 1/2 or any uniform model).  With units of
// q/4, a row is  y_r = (q/4) (D(s_r) x_r + sum over flipped b of 2 k_b x_c),
// D(s) = sum_b k_b eps_b(s) an integer.  x is scaled by 2^S and rounded to
// 64-bit integers X (|X| < 2^B, B chosen so that no row sum can overflow);
// every sum is then exact in integer arithmetic, and each row is converted
// to FP64 once.  The only error is the rounding of x to the 2^-S grid
// (relative 2^-B of the largest entry).
//
// Double-float (any couplings).  x is scaled by a power of two 2^(1023 - E)
// (E the largest biased exponent in x) and split into float pairs
// (hi, lo): hi = the top 24 significant bits of the scaled value (exact), lo
// = the next bits rounded to FP32, |x_s - hi - lo| <= 2^-47 |x_s|.  Each
// coefficient c is a pair (C, gamma), C = fl32(c), gamma = fl32(c - C).  Per
// element, c x is p + e exactly plus the small terms C lo + gamma hi, p =
// fl32(C hi), e = fma(C, hi, -p) (the error-free product of the FMA); p is
// added to the row's accumulator s by TwoSum (Knuth), whose exact rounding
// error joins e and the small terms in the second word.  The row's result
// 2^(E - 1023) (s + c) is formed by integer operations and one FP64
// addition: a relative error near 2^-45 of the sum of the magnitudes of the
// row's terms.
//
// Both arithmetics keep x of one product in a workspace of 8 bytes per row
// (allocated on first use; when it does not fit, the FP64 product falls
// back to the FP64 kernels).

#include <algorithm>
#include <numeric>
#include <vector>

#include "xd_internal.cuh"
#include "xd_layout.h"

namespace xd {

namespace {

constexpr int kB = 8;                 // prefix blocks per work item (the layout's items)
constexpr int kT = 512;               // threads per CTA
constexpr int kPB = 8;                // prefix bonds per step of the prefix streams
constexpr int kL = 12;                // postfix width of the batched layout (N >= 24)
constexpr uint32_t kNlo = 1u << kL;
constexpr int kMB = 924;              // largest block, C(12, 6)
constexpr int kK = (kMB + kT - 1) / kT;  // rows per thread
constexpr uint32_t kEmpty = 0xffffffffu;

struct X64Params {
    int nup;
    const int64_t *hi_off;      // [2^P + 1]
    const uint32_t *lo_off;     // [L + 2]
    const uint32_t *lo_list;    // [2^L]
    const uint32_t *lo_rank;    // [2^L] rank of an L-bit word in its class
    const uint32_t *items;      // [nitems][kB]
    int64_t nitems;
    const uint16_t *xtab;       // [nslot][2^L]
    const int64_t *pcsr_off;    // [2^P + 1] active prefix bonds per prefix
    const uint64_t *pcsr;       // (neighbour block row offset << 12) | bond id
    int maxpa;
    const int32_t *pre;         // [npre][3] prefix bit a, prefix bit b, bond id
    int npre;
    const int32_t *cross;       // [ncross][4] prefix bit, postfix site, bond id, slot
    int ncross;
    const int32_t *csite;       // [ncsite][3] prefix bit, first, end
    int ncsite;
    const uint32_t *post;       // [npost] postfix bond masks (bits i, j of the L-bit word) | bond << 16
    int npost;
    const void *coef;           // [nb] flip coefficient of each bond (the arithmetic's type)
    const void *dpost;          // [2^L] postfix diagonal by class position (the arithmetic's type)
    const void *bdiag;          // [nb] diagonal weight of each bond: J/4 (double) or k_b (int)
    int nb;
    double dcross_d;            // sum over cross bonds of J/4 (double-float)
    int dcross_i;               // sum over cross bonds of k_b (fixed point)
    double qs;                  // q/4 (fixed point)
    int B;                      // |X| < 2^B (fixed point)
    const int *escale;          // [E, mode]: largest biased exponent of x (2047 = x not finite), 1 = fixed point
};

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// A staged row is kB 8-byte values (64 bytes, four 16-byte chunks; chunk j
// holds blocks 2j and 2j + 1).  Chunks are rotated by (row >> 1) & 3 so that
// reads of one block over consecutive rows, and 16-byte reads of whole
// rows, spread over the banks.
__device__ __forceinline__ int swz(int r, int k) {
    return r * kB + ((((k >> 1) ^ (r >> 1)) & 3) << 1) + (k & 1);
}

template <typename V>
__device__ __forceinline__ void row_vals(const V *base, int r, V (&v)[kB]) {
    static_assert(sizeof(V) == 8, "staged values are 8 bytes");
    const int4 *b4 = (const int4 *)(base + r * kB);
    const int s = (r >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int4 q = b4[j ^ s];
        const V *pv = (const V *)&q;
        v[2 * j] = pv[0];
        v[2 * j + 1] = pv[1];
    }
}

// ------------------------------------------------------ double-float pieces
// (s, c) += (C + gamma) (hi + lo): exact product of the leading parts,
// TwoSum into s, every rounding error and the small terms into c.
__device__ __forceinline__ void df_fma(float &s, float &c, float2 C, float2 v) {
    const float p = __fmul_rn(C.x, v.x);
    const float e = __fmaf_rn(C.x, v.x, -p);
    const float low = __fmaf_rn(C.y, v.x, __fmaf_rn(C.x, v.y, e));
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, low));
}

// a - b and a + b for pairs: TwoSum of the leading parts, the rest into the low part
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) {
    const float t = __fsub_rn(a.x, b.x);
    const float bp = __fsub_rn(t, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bp)), __fsub_rn(-b.x, bp));
    return make_float2(t, __fadd_rn(err, __fsub_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float t = __fadd_rn(a.x, b.x);
    const float bp = __fsub_rn(t, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bp)), __fsub_rn(b.x, bp));
    return make_float2(t, __fadd_rn(err, __fadd_rn(a.y, b.y)));
}

// the double 2^(E - 1023) f, built from the bits of f (exact; subnormal f
// is taken as zero); E must keep the result in the normal double range
__device__ __forceinline__ double f2d_scaled(float f, int E) {
    const uint32_t u = __float_as_uint(f);
    const int fe = (int)((u >> 23) & 0xffu);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (fe == 0) return __longlong_as_double((long long)sign);
    return __longlong_as_double((long long)(sign | ((uint64_t)(fe - 127 + E) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}

// 2^(E - 1023) (s + c).  For 300 <= E <= 1700 both words fold the scale into
// their exponents exactly (every float exponent stays inside the normal
// double range) and one FP64 addition rounds the sum.  Otherwise (vectors
// near the ends of the double range) the unscaled sum is multiplied by
// 2^(E - 1023) in FP64, which rounds correctly into the subnormal range or
// to infinity.  E = 2047 (x not finite) gives NaN.
__device__ __forceinline__ double df_result(float s, float c, int E) {
    if (E >= 300 && E <= 1700) return f2d_scaled(s, E) + f2d_scaled(c, E);
    if (E == 2047) return __longlong_as_double(0x7ff8000000000000ll);
    const double v = f2d_scaled(s, 1023) + f2d_scaled(c, 1023);
    return v * __longlong_as_double((long long)((uint64_t)E << 52));
}

__device__ __forceinline__ float2 split_double(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

// 2^k as a double for any k (two factors when 2^k is outside the normal range)
__device__ __forceinline__ double pow2d(int k, double v) {
    if (k >= -1022 && k <= 1023) return v * __longlong_as_double((long long)((uint64_t)(k + 1023) << 52));
    const int h = k / 2;
    v *= __longlong_as_double((long long)((uint64_t)(h + 1023) << 52));
    return v * __longlong_as_double((long long)((uint64_t)(k - h + 1023) << 52));
}

// ------------------------------------------------------------- arithmetics
struct PolDF {
    static constexpr int kMode = 0;
    using V = float2;     // scaled x as (hi, lo)
    using C = float2;     // flip coefficient J/2 as (C, gamma)
    using D = float2;     // diagonal as (C, gamma)
    using DA = double;    // per-block diagonal sum (once per block, FP64)
    struct Acc {
        float s, c;
    };
    struct Out {
        int E;
    };
    __device__ static void zero(Acc &a) { a.s = a.c = 0.f; }
    __device__ static V zero_v() { return make_float2(0.f, 0.f); }
    __device__ static C zero_c() { return make_float2(0.f, 0.f); }
    __device__ static void add(Acc &a, C c, V v) { df_fma(a.s, a.c, c, v); }
    __device__ static void add_diff(Acc &a, C c, V nv, V xv) { df_fma(a.s, a.c, c, df_sub(nv, xv)); }
    __device__ static DA bond_diag(const X64Params &p, int b) { return __ldg((const double *)p.bdiag + b); }
    __device__ static D block_diag(const X64Params &p, DA d) { return split_double(d + p.dcross_d); }
    __device__ static Out out_setup(const X64Params &p, int E) { return Out{E}; }
    __device__ static double result(Acc a, D dpre, D dpost, V xv, const Out &o) {
        df_fma(a.s, a.c, df_add(dpre, dpost), xv);
        return df_result(a.s, a.c, o.E);
    }
};

struct PolFX {
    static constexpr int kMode = 1;
    using V = long long;  // round(2^S x)
    using C = int;        // 2 k_b, in units of q/4
    using D = int;        // D(s) = sum_b k_b eps_b, in units of q/4
    using DA = int;
    struct Acc {
        long long a;
    };
    struct Out {
        double f;         // (q/4) 2^-S
        bool nan;
    };
    __device__ static void zero(Acc &a) { a.a = 0; }
    __device__ static V zero_v() { return 0; }
    __device__ static C zero_c() { return 0; }
    __device__ static void add(Acc &a, C c, V v) { a.a += (long long)c * v; }
    __device__ static void add_diff(Acc &a, C c, V nv, V xv) { a.a += (long long)c * (nv - xv); }
    __device__ static DA bond_diag(const X64Params &p, int b) { return __ldg((const int *)p.bdiag + b); }
    __device__ static D block_diag(const X64Params &p, DA d) { return d + p.dcross_i; }
    __device__ static Out out_setup(const X64Params &p, int E) {
        // S = B - E + 1022: the scaled largest entry is below 2^B
        return Out{pow2d(E - 1022 - p.B, p.qs), E == 2047};
    }
    __device__ static double result(Acc a, D dpre, D dpost, V xv, const Out &o) {
        if (o.nan) return __longlong_as_double(0x7ff8000000000000ll);
        const long long T = a.a + (long long)(dpre + dpost) * xv;
        return (double)T * o.f;
    }
};

template <class Pol>
struct X64Smem {
    size_t xs, nb, cf, pc, pl, plc, cmeta, cc, rqm, noff, nn, lr, pm, total;
    __host__ __device__ X64Smem(const X64Params &p) {
        using V = typename Pol::V;
        using C = typename Pol::C;
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;  // (kMB + 1) rows of kB values
        o += (size_t)(kMB + 1) * kB * sizeof(V);
        al(16);
        nb = o;  // two staging buffers for cross sites
        o += 2 * (size_t)(kMB + 1) * kB * sizeof(V);
        al(16);
        cf = o;
        o += (size_t)p.nb * sizeof(C);
        al(16);
        pc = o;
        o += (size_t)p.npost * sizeof(C);
        al(16);
        pl = o;
        o += (size_t)kB * p.maxpa * sizeof(uint64_t);
        al(16);
        plc = o;  // coefficients of the listed bonds, zero-padded to kPB
        o += (size_t)kB * ((p.maxpa + kPB - 1) / kPB * kPB) * sizeof(C);
        al(16);
        cmeta = o;
        o += (size_t)p.ncross * sizeof(uint32_t);
        al(16);
        cc = o;
        o += (size_t)p.ncross * sizeof(C);
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
        lr = o;  // rank of every L-bit word in its class
        o += (size_t)kNlo * sizeof(uint16_t);
        al(16);
        pm = o;  // postfix bond masks
        o += (size_t)p.npost * sizeof(uint32_t);
        al(16);
        total = o;
    }
};

template <class Pol>
__global__ void __launch_bounds__(kT, 1) k_spmm64(X64Params p, const typename Pol::V *__restrict__ x,
                                                 double *__restrict__ y) {
    using V = typename Pol::V;
    using C = typename Pol::C;
    using D = typename Pol::D;
    using Acc = typename Pol::Acc;
    constexpr int K = kK;
    extern __shared__ __align__(16) unsigned char smem[];
    const X64Smem<Pol> lay(p);
    V *xs = (V *)(smem + lay.xs);
    V *nbuf = (V *)(smem + lay.nb);
    constexpr int NBS = (kMB + 1) * kB;  // values per staging buffer
    C *cf = (C *)(smem + lay.cf);
    C *pc = (C *)(smem + lay.pc);
    uint64_t *pl = (uint64_t *)(smem + lay.pl);
    C *plc = (C *)(smem + lay.plc);
    const int mpc = (p.maxpa + kPB - 1) / kPB * kPB;
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);  // postfix site j | slot << 8
    C *cc = (C *)(smem + lay.cc);                      // flip coefficient of each cross bond
    uint32_t *rqm = (uint32_t *)(smem + lay.rqm);      // per site: bit k = row bit that flips block k
    int64_t *noff = (int64_t *)(smem + lay.noff);
    int *nn = (int *)(smem + lay.nn);
    uint16_t *lr = (uint16_t *)(smem + lay.lr);
    uint32_t *pm = (uint32_t *)(smem + lay.pm);
    __shared__ int sh_npa[kB];
    __shared__ D sh_dpre[kB];
    __shared__ int64_t sh_off[kB];

    // both arithmetics are launched; the one the conversion did not choose returns
    if (__ldg(p.escale + 1) != Pol::kMode) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = tid & (kB - 1);  // staging column of this thread
    const typename Pol::Out oset = Pol::out_setup(p, __ldg(p.escale));
    const C *gcoef = (const C *)p.coef;
    for (int k = tid; k < p.nb; k += kT) cf[k] = gcoef[k];
    for (int k = tid; k < p.npost; k += kT) {
        const uint32_t e = p.post[k];
        pm[k] = e & 0xffffu;
        pc[k] = gcoef[e >> 16];
    }
    for (int q = tid; q < p.ncross; q += kT) {
        cmeta[q] = (uint32_t)p.cross[4 * q + 1] | ((uint32_t)p.cross[4 * q + 3] << 8);
        cc[q] = gcoef[p.cross[4 * q + 2]];
    }
    for (int g = tid; g < (int)kNlo; g += kT) lr[g] = (uint16_t)__ldg(p.lo_rank + g);

    for (int64_t t = blockIdx.x; t < p.nitems; t += gridDim.x) {
        uint32_t hk[kB];
#pragma unroll
        for (int k = 0; k < kB; ++k) hk[k] = __ldg(p.items + t * kB + k);
        const int m = p.nup - __popc(hk[0]);
        const uint32_t l0 = __ldg(p.lo_off + m);
        const int n = (int)(__ldg(p.lo_off + m + 1) - l0);
        const int nm = m > 0 ? (int)(l0 - __ldg(p.lo_off + m - 1)) : 0;
        const int np = m < kL ? (int)(__ldg(p.lo_off + m + 2) - __ldg(p.lo_off + m + 1)) : 0;
        __syncthreads();  // previous item done with shared memory
        {
            const uint32_t hc = hk[col];
            const int64_t offc = hc != kEmpty ? __ldg(p.hi_off + hc) : 0;
            for (int e = tid; e < n * kB; e += kT) {
                const int rr = e >> 3;
                if (hc != kEmpty) cp_async8(xs + swz(rr, col), x + offc + rr);
                else xs[swz(rr, col)] = Pol::zero_v();
            }
            cp_commit();
        }
        if (warp < kB) {
            // per-block data: active prefix bonds, prefix diagonal (once per
            // block), cross neighbour blocks
            const int k = warp;
            const uint32_t h = hk[k];
            typename Pol::DA dpre = 0;
            int cnt = 0;
            if (h != kEmpty) {
                const int64_t c0 = __ldg(p.pcsr_off + h), c1 = __ldg(p.pcsr_off + h + 1);
                cnt = (int)(c1 - c0);
                for (int q = lane; q < (cnt + kPB - 1) / kPB * kPB; q += 32) {
                    const uint64_t ev = q < cnt ? __ldg(p.pcsr + c0 + q) : 0ull;
                    if (q < cnt) pl[k * p.maxpa + q] = ev;
                    plc[k * mpc + q] = q < cnt ? cf[(uint32_t)(ev & 4095u)] : Pol::zero_c();
                }
                for (int q = lane; q < p.npre; q += 32) {
                    const int a = p.pre[3 * q], b = p.pre[3 * q + 1];
                    const typename Pol::DA w = Pol::bond_diag(p, p.pre[3 * q + 2]);
                    dpre += (((h >> a) ^ (h >> b)) & 1u) ? -w : w;
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
                sh_dpre[k] = Pol::block_diag(p, dpre);
                sh_off[k] = h != kEmpty ? __ldg(p.hi_off + h) : 0;
            }
        }
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

        Acc acc[K][kB];
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
            for (int k = 0; k < kB; ++k) Pol::zero(acc[r][k]);
        uint32_t lw[K];
#pragma unroll
        for (int r = 0; r < K; ++r) lw[r] = __ldg(p.lo_list + l0 + min(tid + r * kT, n - 1));

        // postfix bonds: each row walks its own list of flipping bonds (a
        // warp runs as long as its longest list); the target rank comes from
        // the rank table and serves the kB blocks
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT;
            if (i < n) {
                const uint32_t l = lw[r];
#pragma unroll 1
                for (int b0 = 0; b0 < p.npost; b0 += 32) {
                    uint32_t fl = 0;
                    const int bn = min(32, p.npost - b0);
                    for (int b = 0; b < bn; ++b) {
                        const uint32_t mb = pm[b0 + b], t = l & mb;
                        fl |= (uint32_t)(t != 0 && t != mb) << b;
                    }
#pragma unroll 1
                    while (fl) {
                        const int b = __ffs(fl) - 1;
                        fl &= fl - 1;
                        V tv[kB];
                        row_vals(xs, (int)lr[l ^ pm[b0 + b]], tv);
                        const C c = pc[b0 + b];
#pragma unroll
                        for (int k = 0; k < kB; ++k) Pol::add(acc[r][k], c, tv[k]);
                    }
                }
            }
        }
        auto stage_site = [&](int c, V *dst) {
            const int64_t so = noff[c * kB + col];
            const int sn = nn[c * kB + col];
            for (int e = tid; e < sn * kB; e += kT) cp_async8(dst + swz(e >> 3, col), x + so + (e >> 3));
            cp_commit();
        };
        if (p.ncsite > 0) stage_site(0, nbuf);
        // prefix bonds: per block, coalesced streams from its neighbour
        // blocks, kPB neighbours loaded before any use
#pragma unroll
        for (int k = 0; k < kB; ++k) {
            const int npa = sh_npa[k];
            const uint64_t *e = pl + k * p.maxpa;
            const C *cfk = plc + k * mpc;
#pragma unroll 1
            for (int q0 = 0; q0 < npa; q0 += kPB) {
                V v[K][kPB];
#pragma unroll
                for (int w = 0; w < kPB; ++w) {
                    const bool ok = q0 + w < npa;
                    const V *src = x + (ok ? (int64_t)(e[q0 + w] >> 12) : 0);
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        const int i = tid + r * kT;
                        v[r][w] = (ok && i < n) ? __ldg(src + i) : Pol::zero_v();
                    }
                }
#pragma unroll
                for (int w = 0; w < kPB; ++w) {
                    const C c = cfk[q0 + w];
#pragma unroll
                    for (int r = 0; r < K; ++r) Pol::add(acc[r][k], c, v[r][w]);
                }
            }
        }
        // cross bonds: one prefix site at a time, its kB neighbour blocks
        // staged; a flip adds (J/2) (x_target - x_row), which also takes J/2
        // off the diagonal's +J/4 for this bond
#pragma unroll 1
        for (int c = 0; c < p.ncsite; ++c) {
            V *nb = nbuf + (c & 1) * NBS;
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
                    V xv[kB];
                    row_vals(xs, i, xv);
#pragma unroll 1
                    for (int q = q0; q < q1; ++q) {
                        const uint32_t meta = cmeta[q];
                        const uint32_t fm = ((l >> (meta & 31u)) & 1u) ? m1 : m0;
                        if (fm) {
                            const uint32_t r2 = __ldg(p.xtab + (meta >> 8) * kNlo + (l0 + i));
                            const C cq = cc[q];
                            V nv[kB];
                            row_vals(nb, (int)r2, nv);
#pragma unroll
                            for (int k = 0; k < kB; ++k)
                                if ((fm >> k) & 1u) Pol::add_diff(acc[r][k], cq, nv[k], xv[k]);
                        }
                    }
                }
            }
        }
        // diagonal, result in FP64 and store (coalesced per block)
        const D *dpost = (const D *)p.dpost;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT;
            if (i < n) {
                const D dp = dpost[l0 + i];
                V xv[kB];
                row_vals(xs, i, xv);
#pragma unroll
                for (int k = 0; k < kB; ++k)
                    if (hk[k] != kEmpty) y[sh_off[k] + i] = Pol::result(acc[r][k], sh_dpre[k], dp, xv[k], oset);
            }
        }
    }
}

// 4^d for d <= 0 in FP32 (0 below the normal range)
__device__ __forceinline__ float pow4f(int d) { return 2 * d >= -126 ? __uint_as_float((uint32_t)(127 + 2 * d) << 23) : 0.f; }

struct ExpSum {
    int m;    // largest biased exponent seen
    float s;  // sum over the entries seen of 4^(e - m), e their biased exponents
};

__device__ __forceinline__ ExpSum es_join(ExpSum a, ExpSum b) {
    if (a.m == 2047 || b.m == 2047) return ExpSum{2047, 0.f};
    const int m = max(a.m, b.m);
    return ExpSum{m, a.s * pow4f(a.m - m) + b.s * pow4f(b.m - m)};
}

__device__ ExpSum es_block_reduce(ExpSum v) {
    __shared__ ExpSum red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ExpSum w;
        w.m = __shfl_xor_sync(0xffffffffu, v.m, o);
        w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
        v = es_join(v, w);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? red[lane] : ExpSum{0, 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ExpSum w;
            w.m = __shfl_xor_sync(0xffffffffu, v.m, o);
            w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
            v = es_join(v, w);
        }
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    return red[0];
}

// Per CTA: the largest biased exponent of its entries of x (2047 when one is
// infinite or NaN) and sum 4^(e - m) over them, which bounds |x|^2 from
// below within a factor of 4 (zero and subnormal entries count as zero).
__global__ void k_x64_stats(const unsigned long long *__restrict__ x, int64_t n, ExpSum *__restrict__ part) {
    ExpSum v{0, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)((__ldg(x + i) >> 52) & 0x7ffull);
        if (e == 0) continue;
        if (e == 2047) v.m = 2047;
        if (v.m == 2047) continue;
        if (e > v.m) {
            v.s = v.s * pow4f(v.m - e) + 1.f;
            v.m = e;
        } else {
            v.s += pow4f(e - v.m);
        }
    }
    v = es_block_reduce(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

// Every CTA joins the partials into E (largest biased exponent) and S, and
// takes the same decision: fixed point when allowed (the couplings have a
// quantum) and when rounding x to the grid 2^-S of the fixed point, at most
// sqrt(dim) 2^(E - 1023 - B) in norm, stays below 2^-44 |x| with |x|^2 >=
// 4^(E - 1023) S, i.e. dim / S <= 4^(B - 44); else double-float.  CTA 0
// records E and the decision for the product kernels; then x is converted
// (fixed point: X = round(2^S x), S = B - E + 1022, |X| < 2^B; double-float:
// (hi, lo) of 2^(1023 - E) x, hi the top 24 significant bits, lo the next 29
// rounded to FP32).  Subnormal doubles become zero in both.
__global__ void k_x64_convert(const unsigned long long *__restrict__ x, int64_t n, const ExpSum *__restrict__ part,
                              int npart, int fx_allowed, int B, int *__restrict__ state, void *__restrict__ out) {
    ExpSum v{0, 0.f};
    for (int c = threadIdx.x; c < npart; c += blockDim.x) v = es_join(v, part[c]);
    v = es_block_reduce(v);
    const int E = v.m;
    const bool fx = fx_allowed && E != 2047 && E != 0 &&
                    (double)n <= (double)v.s * ldexp(1.0, 2 * (B - 44));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        state[0] = E;
        state[1] = fx ? 1 : 0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = __ldg(x + i);
        const int e = (int)((b >> 52) & 0x7ffull);
        if (fx) {
            long long w = 0;
            if (e != 0) {
                const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
                const int sh = e - E + B - 53;  // 2^S x = M 2^sh, sh <= B - 53
                if (sh >= 0) w = (long long)(M << sh);
                else if (sh > -64) w = (long long)((M >> (-sh)) + ((M >> (-sh - 1)) & 1ull));
                if (b >> 63) w = -w;
            }
            ((long long *)out)[i] = w;
        } else {
            const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
            const int fe = e - E + 127;  // FP32 exponent field of the scaled value
            float hi = 0.f, lo = 0.f;
            if (e != 0 && e != 2047 && fe > 0) {
                hi = __uint_as_float(sign | ((uint32_t)fe << 23) | (uint32_t)((b >> 29) & 0x7fffffull));
                const uint32_t r = (uint32_t)(b & 0x1fffffffull);  // value r 2^(fe - 127 - 52)
                if (r != 0 && fe - 52 > 0)
                    lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(r) *
                                                                __uint_as_float((uint32_t)(fe - 52) << 23)));
            }
            ((float2 *)out)[i] = make_float2(hi, lo);
        }
    }
}

}  // namespace

// Couplings as small integer multiples of one quantum: J_b = k_b q.  With
// J_b = m_b 2^e_b (m_b odd), q = gcd(m) 2^(min e); accepted when every |k_b|
// <= 2^16 and sum |k_b| <= 1365 (so that B >= 47).
static bool find_quantum(const std::vector<double> &J, double *q, std::vector<int> *k) {
    int64_t g = 0;
    int emin = 1 << 20;
    std::vector<std::pair<int64_t, int>> me;
    for (double v : J) {
        if (v == 0.0) {
            me.push_back({0, 0});
            continue;
        }
        int e = 0;
        const double f = frexp(v, &e);             // v = f 2^e, 0.5 <= |f| < 1
        int64_t mm = (int64_t)ldexp(f, 53);        // exact: 53-bit integer
        e -= 53;
        while ((mm & 1) == 0) {
            mm /= 2;
            ++e;
        }
        me.push_back({mm, e});
        g = std::gcd(g, mm < 0 ? -mm : mm);
        emin = std::min(emin, e);
    }
    k->assign(J.size(), 0);
    if (g == 0) {
        *q = 1.0;
        return true;
    }
    int64_t kabs = 0;
    for (size_t b = 0; b < J.size(); ++b) {
        if (me[b].first == 0) continue;
        const int sh = me[b].second - emin;
        const int64_t mq = me[b].first / g;
        if (sh > 16 || mq > 65536 || mq < -65536) return false;
        const int64_t kb = mq * ((int64_t)1 << sh);
        if (kb > 65536 || kb < -65536) return false;
        (*k)[b] = (int)kb;
        kabs += kb < 0 ? -kb : kb;
        if (kabs > 1365) return false;
    }
    *q = ldexp((double)g, emin);
    return true;
}

xd_status spmm64_tables(xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    const int nb = b->nb;
    const uint32_t nlo = 1u << s.L;
    double q = 1.0;
    std::vector<int> k;
    h->x64_fx_ok = find_quantum(h->J, &q, &k);
    std::vector<uint32_t> post(std::max(1, s.npost));
    for (int t = 0; t < s.npost; ++t) {
        const int bd = s.post[t];
        post[t] = (1u << b->bonds[bd].i) | (1u << b->bonds[bd].j) | ((uint32_t)bd << 16);
    }
    auto parity = [&](uint32_t l, int bd) { return ((l >> b->bonds[bd].i) & 1) == ((l >> b->bonds[bd].j) & 1); };
    // double-float tables: J/2 and J/4 per bond, postfix diagonal per class position
    auto pair = [](double d) {
        const float c = (float)d;
        return make_float2(c, (float)(d - (double)c));
    };
    std::vector<float2> dfc(std::max(1, nb)), dfp(nlo);
    std::vector<double> dfd(std::max(1, nb));
    for (int t = 0; t < nb; ++t) {
        dfc[t] = pair(0.5 * h->J[t]);
        dfd[t] = 0.25 * h->J[t];
    }
    for (uint32_t g = 0; g < nlo; ++g) {
        double d = 0.0;
        for (int bd : s.post) d += (parity(s.h_lo_list[g], bd) ? 0.25 : -0.25) * h->J[bd];
        dfp[g] = pair(d);
    }
    double dcd = 0.0;
    for (int bd : s.cross_ids) dcd += 0.25 * h->J[bd];
    h->x64_dcross_d = dcd;
    // fixed-point tables: 2 k_b and k_b per bond, postfix D per class position
    std::vector<int> fxc(std::max(1, nb), 0), fxd(std::max(1, nb), 0), fxp(nlo, 0);
    if (h->x64_fx_ok) {
        int64_t kabs = 0;
        for (int t = 0; t < nb; ++t) {
            fxc[t] = 2 * k[t];
            fxd[t] = k[t];
            kabs += std::abs(k[t]);
        }
        for (uint32_t g = 0; g < nlo; ++g) {
            int d = 0;
            for (int bd : s.post) d += parity(s.h_lo_list[g], bd) ? k[bd] : -k[bd];
            fxp[g] = d;
        }
        int dci = 0;
        for (int bd : s.cross_ids) dci += k[bd];
        h->x64_dcross_i = dci;
        h->x64_qs = 0.25 * q;
        // every row sum is at most 3 sum|k_b| max|X| < 2^62
        int lg = 0;
        while ((int64_t(1) << lg) < 3 * std::max<int64_t>(1, kabs)) ++lg;
        h->x64_B = 62 - lg;
    }
    const size_t cb = (size_t)std::max(1, nb) * 8, pb = (size_t)nlo * 8;
    if (!h->d_x64_tab) {
        XD_CUDA(dev_malloc(&h->d_x64_tab, 6 * std::max(cb, pb) + post.size() * sizeof(uint32_t)));
    }
    unsigned char *base = (unsigned char *)h->d_x64_tab;
    const size_t st = std::max(cb, pb);
    h->d_x64_dfc = base;
    h->d_x64_dfd = base + st;
    h->d_x64_dfp = base + 2 * st;
    h->d_x64_fxc = base + 3 * st;
    h->d_x64_fxd = base + 4 * st;
    h->d_x64_fxp = base + 5 * st;
    h->d_x64_post = (uint32_t *)(base + 6 * st);
    XD_CUDA(cudaMemcpy(h->d_x64_dfc, dfc.data(), dfc.size() * sizeof(float2), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_dfd, dfd.data(), dfd.size() * sizeof(double), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_dfp, dfp.data(), dfp.size() * sizeof(float2), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_fxc, fxc.data(), fxc.size() * sizeof(int), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_fxd, fxd.data(), fxd.size() * sizeof(int), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_fxp, fxp.data(), fxp.size() * sizeof(int), cudaMemcpyHostToDevice));
    XD_CUDA(cudaMemcpy(h->d_x64_post, post.data(), post.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    return XD_OK;
}

constexpr int kStatThreads = 256;
constexpr int kStatPerSm = 8;

// The workspace (8 bytes per row, the two state words and the partials of
// the statistics pass) is allocated on first use.  When it does not fit, the
// call returns XD_ENOMEM and this product takes the FP64 kernels; the next
// product tries again (the drivers that hold several vectors release the
// workspace when their own vectors do not fit, x64_release).
static xd_status x64_workspace(xd_ham_s *h, int64_t dim) {
    grid_for(1, 1, 1);
    if (!h->d_x64_state) {
        cudaError_t e = dev_malloc((void **)&h->d_x64_state, 16 + (size_t)g_num_sms * kStatPerSm * sizeof(ExpSum));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return XD_ENOMEM;
        }
    }
    if (h->d_x64_x) return XD_OK;
    cudaError_t e = dev_malloc((void **)&h->d_x64_x, (size_t)dim * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->d_x64_x = nullptr;
        return XD_ENOMEM;
    }
    return XD_OK;
}

void x64_release(xd_ham_s *h) {
    if (h->d_x64_x) {
        cudaFree(h->d_x64_x);
        h->d_x64_x = nullptr;
    }
}

template <class Pol>
static xd_status launch64(const xd_ham_s *h, void *y, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    const bool fx = Pol::kMode == 1;
    X64Params p;
    p.nup = b->nup;
    p.hi_off = s.d_hi_off;
    p.lo_off = s.d_lo_off;
    p.lo_list = s.d_lo_list;
    p.lo_rank = s.d_lo_rank;
    p.items = s.d_items;
    p.nitems = s.nitems;
    p.xtab = s.d_xtab;
    p.pcsr_off = s.d_pcsr_off;
    p.pcsr = s.d_pcsr;
    p.maxpa = s.maxpa;
    p.pre = s.d_pre;
    p.npre = s.npre;
    p.cross = s.d_cross;
    p.ncross = s.ncross;
    p.csite = s.d_csite;
    p.ncsite = s.ncsite;
    p.post = h->d_x64_post;
    p.npost = s.npost;
    p.coef = fx ? h->d_x64_fxc : h->d_x64_dfc;
    p.dpost = fx ? h->d_x64_fxp : h->d_x64_dfp;
    p.bdiag = fx ? h->d_x64_fxd : h->d_x64_dfd;
    p.nb = b->nb;
    p.dcross_d = h->x64_dcross_d;
    p.dcross_i = h->x64_dcross_i;
    p.qs = h->x64_qs;
    p.B = h->x64_B;
    p.escale = h->d_x64_state;
    const X64Smem<Pol> lay(p);
    auto kern = k_spmm64<Pol>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, lay.total));
    if (per_sm < 1) {
        set_error("FP64 product: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    grid_for(1, 1, 1);
    const int grid = (int)std::min<int64_t>(s.nitems, (int64_t)g_num_sms * per_sm);
    kern<<<grid, kT, lay.total, st>>>(p, (const typename Pol::V *)h->d_x64_x, (double *)y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// the batched layout has L = 12 for every block it is built for (N >= 24)
bool spmm64_usable(const xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    return b->spmm.ok && b->spmm.L == kL && h->d_x64_tab != nullptr;
}

// Statistics of x, the choice of arithmetic and the conversion on the
// device; both product kernels are launched and the one not chosen returns
// at once (no host synchronisation).
xd_status spmm64_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    xd_ham_s *hm = const_cast<xd_ham_s *>(h);
    const int64_t dim = h->b->dim;
    XD_TRY(x64_workspace(hm, dim));
    const int g1 = grid_for(dim, kStatThreads, kStatPerSm);
    ExpSum *part = (ExpSum *)((unsigned char *)h->d_x64_state + 16);
    k_x64_stats<<<g1, kStatThreads, 0, st>>>((const unsigned long long *)x, dim, part);
    k_x64_convert<<<g1, kStatThreads, 0, st>>>((const unsigned long long *)x, dim, part, g1, h->x64_fx_ok ? 1 : 0,
                                               h->x64_B, h->d_x64_state, h->d_x64_x);
    XD_CUDA(cudaGetLastError());
    if (h->x64_fx_ok) XD_TRY(launch64<PolFX>(h, y, st));
    return launch64<PolDF>(h, y, st);
}

}  // namespace xd

// xd_u1_passes.cu -- FP64 y = H x on large U(1) blocks (N >= 24) in passes
// over prefix blocks, without FP64 arithmetic per matrix element.
//
// With the prefix/postfix split of the index layout (Sec. 5.2 two tables,
// Sec. 5.3 prefix/postfix view) H = H_pre + H_post + H_cross (Eq. 1, pull
// form, rows written once, no atomics):
//   * H_pre maps block h to block h ^ m_b with the same in-block rank.  It
//     runs as passes (k_tpass), each over the prefix bonds inside a window
//     of at most 12 prefix bits (choose_passes, xd_layout.h): rows that
//     share the prefix bits outside the window, the popcount of the window
//     word and a chunk of 8 postfix ranks form a set closed under the pass's
//     flips, staged as one transposed tile in shared memory, so x is read
//     once per pass and every prefix flip is a shared-memory gather (one
//     rank lookup serving 8 ranks).  The passes accumulate into y's memory.
//   * H_post and H_cross run in k_main on work items of KB same-class
//     prefix blocks staged transposed in shared memory (one target rank
//     serves KB blocks), items in an order that keeps the cross neighbour
//     blocks (flips of the prefix sites of cross bonds) in L2.  k_main adds
//     the passes' sums and the diagonal and writes y.
// Arithmetic: FP64 input and output (the paper's precision) without FP64
// arithmetic per element (GB300's FP64 pipe is a small fraction of its FP32
// and integer rates), in one of two arithmetics chosen per product on the
// device:
//     fixed point, for couplings that are small integer multiples k_b q of
//     one quantum q (e.g. J1 = 1, J2 = 1/2, any uniform model): in units of
//     q/4 a row is y_r = (q/4) (D(s_r) x_r + sum over flipped b of 2 k_b x_c),
//     D(s) = sum_b k_b eps_b(s) an integer; x is scaled by 2^S and rounded to
//     64-bit integers X (|X| < 2^B, no row sum can overflow) and every sum
//     is exact; each row is converted to FP64 once;
//     double-float, for any couplings: x is scaled by 2^(1023 - E) (E its
//     largest biased exponent) and split into FP32 pairs (hi, lo), hi the
//     top 24 significant bits (exact), lo the next bits rounded to FP32; each
//     coefficient c is a pair (C, gamma); per element c x is p + e exactly
//     (p = fl32(C hi), e = fma(C, hi, -p)) plus the small terms C lo + gamma
//     hi, p enters the accumulator by TwoSum (Knuth) and every rounding error
//     joins the second word; the row's result 2^(E - 1023) (s + c) costs one
//     FP64 addition: a relative error near 2^-45 of the sum of the
//     magnitudes of the row's terms.
//     A statistics pass (largest exponent and a lower bound of |x|) lets the
//     device take double-float whenever rounding x to the fixed-point grid
//     could cost more than 2^-44 |x| (vectors dominated by a few entries).

#include <algorithm>
#include <numeric>
#include <vector>

#include "xd_internal.cuh"
#include "xd_layout.h"

namespace xd {

namespace {

constexpr int kT = 512;               // threads per CTA of k_main
constexpr int kL = 12;                // postfix width of the batched layout (N >= 24)
constexpr uint32_t kNlo = 1u << kL;
constexpr int kMB = 924;              // largest block, C(12, 6)
constexpr int kK = (kMB + kT - 1) / kT;  // rows per thread
constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ void cp_async_n(void *smem_dst, const void *gsrc, int bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
struct MainParams;

struct PolDF {
    static constexpr int kMode = 0;
    static constexpr bool kFoldCross = false;  // a cross flip adds c (x_target - x_row) in pairs
    using V = float2;     // scaled x as (hi, lo)
    using C = float2;     // flip coefficient J/2 as (C, gamma)
    using D = float2;     // diagonal as (C, gamma)
    using DA = double;    // per-block diagonal sum (once per block, FP64)
    using Y = double;
    struct __align__(8) Acc {
        float s, c;
    };
    struct Out {
        int E;
    };
    __device__ static void zero(Acc &a) { a.s = a.c = 0.f; }
    __device__ static V zero_v() { return make_float2(0.f, 0.f); }
    __device__ static void add(Acc &a, C c, V v) { df_fma(a.s, a.c, c, v); }
    __device__ static void add_diff(Acc &a, C c, V nv, V xv) { df_fma(a.s, a.c, c, df_sub(nv, xv)); }
    __device__ static void merge(Acc &a, Acc b) {
        const float2 r = df_add(make_float2(a.s, a.c), make_float2(b.s, b.c));
        a.s = r.x;
        a.c = r.y;
    }
    __device__ static DA bond_diag(const void *bdiag, const void *, int b) { return __ldg((const double *)bdiag + b); }
    template <class P> __device__ static D block_diag(const P &p, DA d) { return split_double(d + p.dcross_d); }
    template <class P> __device__ static Out out_setup(const P &, int E) { return Out{E}; }
    __device__ static Y result(Acc a, D dpre, D dpost, V xv, const Out &o) {
        df_fma(a.s, a.c, df_add(dpre, dpost), xv);
        return df_result(a.s, a.c, o.E);
    }
};

struct PolFX {
    static constexpr int kMode = 1;
    // a cross flip adds c x_target, and its -c x_row joins the row's integer
    // diagonal (exact: the same integers summed in another order)
    static constexpr bool kFoldCross = true;
    using V = long long;  // round(2^S x)
    using C = int;        // 2 k_b, in units of q/4
    using D = int;        // D(s) = sum_b k_b eps_b, in units of q/4
    using DA = int;
    using Y = double;
    struct Acc {
        long long a;
    };
    struct Out {
        double f;         // (q/4) 2^-S
        bool nan;
    };
    __device__ static void zero(Acc &a) { a.a = 0; }
    __device__ static V zero_v() { return 0; }
    __device__ static void add(Acc &a, C c, V v) { a.a += (long long)c * v; }
    __device__ static void add_diff(Acc &a, C c, V nv, V xv) { a.a += (long long)c * (nv - xv); }
    __device__ static void merge(Acc &a, Acc b) { a.a += b.a; }
    __device__ static DA bond_diag(const void *bdiag, const void *, int b) { return __ldg((const int *)bdiag + b); }
    template <class P> __device__ static D block_diag(const P &p, DA d) { return d + p.dcross_i; }
    template <class P> __device__ static Out out_setup(const P &p, int E) {
        // S = B - E + 1022: the scaled largest entry is below 2^B
        return Out{pow2d(E - 1022 - p.B, p.qs), E == 2047};
    }
    __device__ static Y result(Acc a, D dpre, D dpost, V xv, const Out &o) {
        if (o.nan) return __longlong_as_double(0x7ff8000000000000ll);
        const long long T = a.a + (long long)(dpre + dpost) * xv;
        return (double)T * o.f;
    }
};

// A staged row holds the KB blocks' values of one in-block rank (32 or 64
// bytes, 16-byte chunks).  Chunks are rotated along the rows so that reads of
// one block over consecutive rows, and 16-byte reads of whole rows, spread
// over the banks.
template <typename V, int KB>
struct Rows {
    static constexpr int VPC = 16 / (int)sizeof(V);   // values per chunk
    static constexpr int NCH = KB / VPC;              // chunks per row (2 or 4)
    __device__ static int rot(int r) { return NCH == 4 ? ((r >> 1) & 3) : ((r >> 2) & 1); }
    __device__ static int at(int r, int k) { return r * KB + (((k / VPC) ^ rot(r)) * VPC) + (k % VPC); }
    __device__ static void load(const V *base, int r, V (&v)[KB]) {
        const int4 *b4 = (const int4 *)(base + r * KB);
        const int s = rot(r);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const int4 q = b4[j ^ s];
            const V *pv = (const V *)&q;
#pragma unroll
            for (int t = 0; t < VPC; ++t) v[j * VPC + t] = pv[t];
        }
    }
};

// ------------------------------------------------------------ prefix passes
// A pass takes the prefix bonds whose two bits lie in a window S of at most
// 12 prefix bits (choose_passes, xd_layout.h).  Split a prefix h into its
// window word w (the bits of S) and the rest o: the flips of the pass's
// bonds change w only, keeping its popcount, so the rows (h, q) for one o,
// one popcount k of w and one postfix rank q form a closed set under the
// pass's bonds: a transposed tile [C(|S|, k) words][8 consecutive ranks q] is
// staged in shared memory (x read once per pass), and each row of the tile
// walks its list of flipping bonds, one rank lookup serving 8 ranks -- the
// postfix phase of k_main with the roles of prefix and postfix swapped.
struct TPassParams {
    int nup;
    const int64_t *hi_off;      // [2^P + 1]
    const uint32_t *lo_off;     // [L + 2]
    const uint64_t *items;      // o's deposited prefix bits | k << 32 | rank chunk << 40
    int64_t nitems;
    const uint16_t *wlist;      // [2^ws] window words by (popcount, value)
    const uint32_t *woff;       // [ws + 2] first word of each popcount
    const uint16_t *wrank;      // [2^ws] rank of a window word in its popcount
    const uint32_t *wdep;       // [2^ws] the window word's bits deposited at their prefix bits
    const uint32_t *wbond;      // [nwb] the pass's bonds: window mask | bond << 16
    int nwb, ws;
    const void *coef;           // [nb] flip coefficient of each bond (the arithmetic's type)
    const int *state;           // [E, mode] of the FP64 arithmetics (unused for FP32)
};

constexpr int kTQ = 8;          // postfix ranks per tile

struct TPassSmem {
    size_t at, bo, wr, wm, wc, total;
    __host__ __device__ TPassSmem(int ws, int nwb, size_t vsize, size_t csize, size_t asize, bool first) {
        auto al = [](size_t o) { return (o + 15) / 16 * 16; };
        at = al((size_t)(kMB + 1) * kTQ * vsize);                  // the accumulator tile (later passes)
        bo = al(at + (first ? 0 : (size_t)kMB * kTQ * asize));     // block offset of each tile row
        wr = al(bo + (size_t)kMB * sizeof(int64_t));
        wm = al(wr + ((size_t)1 << ws) * sizeof(uint16_t));
        wc = al(wm + (size_t)nwb * sizeof(uint32_t));
        total = al(wc + (size_t)nwb * csize);
    }
};

template <class Pol, bool FIRST>
__global__ void __launch_bounds__(kT, 2) k_tpass(TPassParams p, const typename Pol::V *__restrict__ x,
                                                typename Pol::Acc *acc) {
    using V = typename Pol::V;
    using C = typename Pol::C;
    using Acc = typename Pol::Acc;
    using R = Rows<V, kTQ>;
    using RA = Rows<Acc, kTQ>;  // the accumulator tile, rotated like the x tile
    constexpr int K = kK;
    if (Pol::kMode >= 0 && __ldg(p.state + 1) != Pol::kMode) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const TPassSmem lay(p.ws, p.nwb, sizeof(V), sizeof(C), sizeof(Acc), FIRST);
    V *tile = (V *)smem;                         // [(kMB + 1) * kTQ] x of the tile, transposed
    Acc *atile = (Acc *)(smem + lay.at);         // [kMB * kTQ] the sums so far (later passes)
    int64_t *bo = (int64_t *)(smem + lay.bo);    // [kMB] first row of the tile row's ranks in x
    uint16_t *wr = (uint16_t *)(smem + lay.wr);  // [2^ws]
    uint32_t *wm = (uint32_t *)(smem + lay.wm);  // [nwb]
    C *wc = (C *)(smem + lay.wc);                // [nwb]
    const int tid = threadIdx.x;
    const C *gcoef = (const C *)p.coef;
    for (int g = tid; g < (1 << p.ws); g += kT) wr[g] = __ldg(p.wrank + g);
    for (int q = tid; q < p.nwb; q += kT) {
        const uint32_t e = p.wbond[q];
        wm[q] = e & 0xffffu;
        wc[q] = gcoef[e >> 16];
    }
    for (int64_t t = blockIdx.x; t < p.nitems; t += gridDim.x) {
        const uint64_t it = __ldg(p.items + t);
        const uint32_t ho = (uint32_t)it;
        const int k = (int)((it >> 32) & 0xffu);
        const int q0 = (int)(it >> 40) * kTQ;
        const uint32_t w0 = __ldg(p.woff + k);
        const int nw = (int)(__ldg(p.woff + k + 1) - w0);
        const int m = p.nup - __popc(ho) - k;
        const int nq = min(kTQ, (int)(__ldg(p.lo_off + m + 1) - __ldg(p.lo_off + m)) - q0);
        __syncthreads();  // previous item done with shared memory
        for (int r = tid; r < nw; r += kT) bo[r] = __ldg(p.hi_off + (ho | __ldg(p.wdep + __ldg(p.wlist + w0 + r)))) + q0;
        __syncthreads();
        for (int e = tid; e < nw * kTQ; e += kT) {
            const int r = e / kTQ, j = e % kTQ;
            if (j < nq) {
                cp_async_n(tile + R::at(r, j), x + bo[r] + j, (int)sizeof(V));
                if (!FIRST) cp_async_n(atile + RA::at(r, j), acc + bo[r] + j, (int)sizeof(Acc));
            } else {
                tile[R::at(r, j)] = Pol::zero_v();
            }
        }
        cp_commit();
        cp_wait_all();
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < K; ++rr) {
            const int r = tid + rr * kT;
            if (r < nw) {
                const uint32_t w = __ldg(p.wlist + w0 + r);
                Acc a[kTQ];
#pragma unroll
                for (int j = 0; j < kTQ; ++j) Pol::zero(a[j]);
#pragma unroll 1
                for (int b0 = 0; b0 < p.nwb; b0 += 32) {
                    uint32_t fl = 0;
                    const int bn = min(32, p.nwb - b0);
                    for (int b = 0; b < bn; ++b) {
                        const uint32_t mb = wm[b0 + b], tq = w & mb;
                        fl |= (uint32_t)(tq != 0 && tq != mb) << b;
                    }
#pragma unroll 1
                    while (fl) {
                        const int b = __ffs(fl) - 1;
                        fl &= fl - 1;
                        V tv[kTQ];
                        R::load(tile, (int)wr[w ^ wm[b0 + b]], tv);
                        const C c = wc[b0 + b];
#pragma unroll
                        for (int j = 0; j < kTQ; ++j) Pol::add(a[j], c, tv[j]);
                    }
                }
                const int64_t base = bo[r];
                Acc prev[kTQ];
                if (!FIRST) RA::load(atile, r, prev);  // 16-byte reads of the rotated row
#pragma unroll
                for (int j = 0; j < kTQ; ++j)
                    if (j < nq) {
                        if (!FIRST) Pol::merge(a[j], prev[j]);
                        acc[base + j] = a[j];
                    }
            }
        }
    }
}

// ----------------------------------------------------- postfix, cross, diagonal
struct MainParams {
    int nup;
    const int64_t *hi_off;      // [2^P + 1]
    const uint32_t *lo_off;     // [L + 2]
    const uint32_t *lo_list;    // [2^L]
    const uint32_t *lo_rank;    // [2^L] rank of an L-bit word in its class
    const uint32_t *items;      // [nitems][KB] same-class prefixes
    int64_t nitems;
    const uint16_t *xtab;       // [nslot][2^L] rank of l ^ 2^j_slot in its class
    const int32_t *pre;         // [npre][3] prefix bit a, prefix bit b, bond id
    int npre;
    const int32_t *cross;       // [ncross][4] prefix bit, postfix site, bond id, slot
    int ncross;
    const int32_t *csite;       // [ncsite][3] prefix bit, first, end
    int ncsite;
    const uint32_t *post;       // [npost] postfix bond masks (bits of the L-bit word) | bond << 16
    int npost;
    const void *coef;           // [nb] flip coefficient of each bond (the arithmetic's type)
    const void *dpost;          // [2^L] postfix diagonal by class position (the arithmetic's type)
    const void *bdiag;          // [nb] diagonal weight of each bond (double-float: J/4; fixed point: k_b)
    int nb;
    double dcross_d;            // same (double-float)
    int dcross_i;               // sum over cross bonds of k_b (fixed point)
    double qs;                  // q/4 (fixed point)
    int B;                      // |X| < 2^B (fixed point)
    const int *state;           // [E, mode] of the FP64 arithmetics
};

template <class Pol, int KB>
struct MainSmem {
    size_t xs, nb, cf, pc, cmeta, cc, rqm, noff, nn, lr, pm, total;
    __host__ __device__ MainSmem(const MainParams &p) {
        using V = typename Pol::V;
        using C = typename Pol::C;
        size_t o = 0;
        auto al = [&](size_t a) { o = (o + a - 1) / a * a; };
        xs = o;  // (kMB + 1) rows of KB values
        o += (size_t)(kMB + 1) * KB * sizeof(V);
        al(16);
        nb = o;  // two staging buffers for cross sites
        o += 2 * (size_t)(kMB + 1) * KB * sizeof(V);
        al(16);
        cf = o;
        o += (size_t)p.nb * sizeof(C);
        al(16);
        pc = o;
        o += (size_t)p.npost * sizeof(C);
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
        o += (size_t)p.ncsite * KB * sizeof(int64_t);
        al(16);
        nn = o;
        o += (size_t)p.ncsite * KB * sizeof(int);
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

template <class Pol, int KB>
__global__ void __launch_bounds__(kT, 2) k_main(MainParams p, const typename Pol::V *__restrict__ x,
                                               const typename Pol::Acc *acc_in, typename Pol::Y *y) {
    using V = typename Pol::V;
    using C = typename Pol::C;
    using D = typename Pol::D;
    using Acc = typename Pol::Acc;
    using R = Rows<V, KB>;
    constexpr int K = kK;
    if (Pol::kMode >= 0 && __ldg(p.state + 1) != Pol::kMode) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const MainSmem<Pol, KB> lay(p);
    V *xs = (V *)(smem + lay.xs);
    V *nbuf = (V *)(smem + lay.nb);
    constexpr int NBS = (kMB + 1) * KB;  // values per staging buffer
    C *cf = (C *)(smem + lay.cf);
    C *pc = (C *)(smem + lay.pc);
    uint32_t *cmeta = (uint32_t *)(smem + lay.cmeta);  // postfix site j | slot << 8
    C *cc = (C *)(smem + lay.cc);                      // flip coefficient of each cross bond
    uint32_t *rqm = (uint32_t *)(smem + lay.rqm);      // per site: bit k = row bit that flips block k
    int64_t *noff = (int64_t *)(smem + lay.noff);
    int *nn = (int *)(smem + lay.nn);
    uint16_t *lr = (uint16_t *)(smem + lay.lr);
    uint32_t *pm = (uint32_t *)(smem + lay.pm);
    __shared__ D sh_dpre[KB];
    __shared__ int64_t sh_off[KB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int col = tid % KB;  // staging column of this thread
    const typename Pol::Out oset = Pol::out_setup(p, Pol::kMode >= 0 ? __ldg(p.state) : 0);
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
        uint32_t hk[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) hk[k] = __ldg(p.items + t * KB + k);
        const int m = p.nup - __popc(hk[0]);
        const uint32_t l0 = __ldg(p.lo_off + m);
        const int n = (int)(__ldg(p.lo_off + m + 1) - l0);
        const int nm = m > 0 ? (int)(l0 - __ldg(p.lo_off + m - 1)) : 0;
        const int np = m < kL ? (int)(__ldg(p.lo_off + m + 2) - __ldg(p.lo_off + m + 1)) : 0;
        __syncthreads();  // previous item done with shared memory
        {
            const uint32_t hc = hk[col];
            const int64_t offc = hc != kEmpty ? __ldg(p.hi_off + hc) : 0;
            for (int e = tid; e < n * KB; e += kT) {
                const int rr = e / KB;
                if (hc != kEmpty) cp_async_n(xs + R::at(rr, col), x + offc + rr, (int)sizeof(V));
                else xs[R::at(rr, col)] = Pol::zero_v();
            }
            cp_commit();
        }
        if (warp < KB) {
            // per-block data: prefix diagonal (once per block), cross neighbour blocks
            const int k = warp;
            const uint32_t h = hk[k];
            typename Pol::DA dpre = 0;
            if (h != kEmpty) {
                for (int q = lane; q < p.npre; q += 32) {
                    const int a = p.pre[3 * q], b = p.pre[3 * q + 1];
                    const typename Pol::DA w = Pol::bond_diag(p.bdiag, p.coef, p.pre[3 * q + 2]);
                    dpre += (((h >> a) ^ (h >> b)) & 1u) ? -w : w;
                }
                for (int c = lane; c < p.ncsite; c += 32) {
                    const int a = p.csite[3 * c];
                    const int hb = (int)((h >> a) & 1u);
                    noff[c * KB + k] = __ldg(p.hi_off + (h ^ (1u << a)));
                    nn[c * KB + k] = hb ? np : nm;
                }
            } else {
                for (int c = lane; c < p.ncsite; c += 32) {
                    noff[c * KB + k] = 0;
                    nn[c * KB + k] = 0;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dpre += __shfl_xor_sync(0xffffffffu, dpre, o);
            if (lane == 0) {
                sh_dpre[k] = Pol::block_diag(p, dpre);
                sh_off[k] = h != kEmpty ? __ldg(p.hi_off + h) : 0;
            }
        }
        for (int c = tid; c < p.ncsite; c += kT) {
            uint32_t m1 = 0;
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (hk[k] != kEmpty && !((hk[k] >> p.csite[3 * c]) & 1u)) m1 |= 1u << k;
            rqm[c] = m1;
        }
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0; k < KB; ++k) valid |= (hk[k] != kEmpty ? 1u : 0u) << k;
        cp_wait_all();
        __syncthreads();

        Acc acc[K][KB];
        C cs[K][KB];  // kFoldCross: the row's sum of the cross flips' coefficients
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                Pol::zero(acc[r][k]);
                cs[r][k] = C();
            }
        uint32_t lw[K];
#pragma unroll
        for (int r = 0; r < K; ++r) lw[r] = __ldg(p.lo_list + l0 + min(tid + r * kT, n - 1));

        // postfix bonds: each row walks its own list of flipping bonds (a
        // warp runs as long as its longest list); the target rank comes from
        // the rank table and serves the KB blocks
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
                        const uint32_t mb = pm[b0 + b], tq = l & mb;
                        fl |= (uint32_t)(tq != 0 && tq != mb) << b;
                    }
#pragma unroll 1
                    while (fl) {
                        const int b = __ffs(fl) - 1;
                        fl &= fl - 1;
                        V tv[KB];
                        R::load(xs, (int)lr[l ^ pm[b0 + b]], tv);
                        const C c = pc[b0 + b];
#pragma unroll
                        for (int k = 0; k < KB; ++k) Pol::add(acc[r][k], c, tv[k]);
                    }
                }
            }
        }
        // cross bonds: one prefix site at a time, its KB neighbour blocks
        // staged (the next site's copy overlaps this site's arithmetic); a
        // flip adds (J/2) (x_target - x_row), which also takes J/2 off the
        // diagonal's +J/4 for this bond
        auto stage_site = [&](int c, V *dst) {
            const int64_t so = noff[c * KB + col];
            const int sn = nn[c * KB + col];
            for (int e = tid; e < sn * KB; e += kT) cp_async_n(dst + R::at(e / KB, col), x + so + e / KB, (int)sizeof(V));
            cp_commit();
        };
        if (p.ncsite > 0) stage_site(0, nbuf);
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
                    V xv[KB];
                    if (!Pol::kFoldCross) R::load(xs, i, xv);
#pragma unroll 1
                    for (int q = q0; q < q1; ++q) {
                        const uint32_t meta = cmeta[q];
                        const uint32_t fm = ((l >> (meta & 31u)) & 1u) ? m1 : m0;
                        if (fm) {
                            const uint32_t r2 = __ldg(p.xtab + (meta >> 8) * kNlo + (l0 + i));
                            const C cq = cc[q];
                            V nv[KB];
                            R::load(nb, (int)r2, nv);
#pragma unroll
                            for (int k = 0; k < KB; ++k)
                                if ((fm >> k) & 1u) {
                                    if constexpr (Pol::kFoldCross) {
                                        Pol::add(acc[r][k], cq, nv[k]);
                                        cs[r][k] += cq;
                                    } else {
                                        Pol::add_diff(acc[r][k], cq, nv[k], xv[k]);
                                    }
                                }
                        }
                    }
                }
            }
        }
        // the passes' prefix sums, the diagonal, the result (coalesced per block)
        const D *dpost = (const D *)p.dpost;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int i = tid + r * kT;
            if (i < n) {
                const D dp = dpost[l0 + i];
                V xv[KB];
                R::load(xs, i, xv);
#pragma unroll
                for (int k = 0; k < KB; ++k)
                    if (hk[k] != kEmpty) {
                        Acc a = acc[r][k];
                        Pol::merge(a, acc_in[sh_off[k] + i]);
                        D dk = sh_dpre[k];
                        if constexpr (Pol::kFoldCross) dk -= cs[r][k];
                        y[sh_off[k] + i] = Pol::result(a, dk, dp, xv[k], oset);
                    }
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

xd_status passes_tables(xd_ham_s *h) {
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

// Passes of the prefix bonds and the work items of k_main for this basis,
// built on first use: windows of at most 12 prefix bits (a tile then holds at
// most C(12, 6) window words), at most four passes.
static xd_status pass_layout_build(xd_basis_s *b) {
    PassLayoutHost &pl = b->pass;
    if (pl.ok) return pl.unusable ? XD_ERANGE : XD_OK;
    const SpmmLayoutHost &s = b->spmm;
    const int P = s.P, L = s.L, nup = b->nup;
    std::vector<PrefixPass> passes = choose_passes(P, s.h_pre, std::min(12, P), 4);
    // a graph whose prefix bonds four windows cannot hold takes the FP64 block kernel
    for (const PrefixPass &ps : passes)
        for (int t : ps.bonds)
            if (std::find(ps.low.begin(), ps.low.end(), s.h_pre[3 * t]) == ps.low.end() ||
                std::find(ps.low.begin(), ps.low.end(), s.h_pre[3 * t + 1]) == ps.low.end()) {
                pl.ok = pl.unusable = true;
                set_error("FP64 product: prefix bonds beyond four windows");
                return XD_ERANGE;
            }
    if (passes.empty()) {
        PrefixPass ps;
        for (int v = 0; v < std::min(12, P); ++v) ps.low.push_back(v);
        passes.push_back(ps);
    }
    pl.npass = (int)passes.size();
    for (int q = 0; q < pl.npass; ++q) {
        const std::vector<int> &S = passes[q].low;
        const int ws = (int)S.size();
        const uint32_t nw = 1u << ws;
        // window words by (popcount, value), their ranks and deposited bits
        std::vector<uint32_t> woff(ws + 2, 0);
        for (int k = 0; k <= ws; ++k) woff[k + 1] = woff[k] + (uint32_t)n_choose_k(ws, k);
        std::vector<uint16_t> wlist(nw), wrank(nw);
        std::vector<uint32_t> wdep(nw), fill(woff.begin(), woff.end() - 1);
        for (uint32_t w = 0; w < nw; ++w) {
            const int k = __builtin_popcount(w);
            wrank[w] = (uint16_t)(fill[k] - woff[k]);
            wlist[fill[k]++] = (uint16_t)w;
            uint32_t d = 0;
            for (int i = 0; i < ws; ++i) d |= ((w >> i) & 1u) << S[i];
            wdep[w] = d;
        }
        std::vector<uint32_t> wb;
        for (int t : passes[q].bonds) {
            const int a = s.h_pre[3 * t], c = s.h_pre[3 * t + 1];
            const int ia = (int)(std::find(S.begin(), S.end(), a) - S.begin());
            const int ic = (int)(std::find(S.begin(), S.end(), c) - S.begin());
            wb.push_back((1u << ia) | (1u << ic) | ((uint32_t)s.h_pre[3 * t + 2] << 16));
        }
        // items: the other prefix bits o, the window popcount k, the chunk of 8 ranks
        std::vector<int> outer;
        for (int v = 0; v < P; ++v)
            if (std::find(S.begin(), S.end(), v) == S.end()) outer.push_back(v);
        std::vector<uint64_t> items;
        for (uint64_t o = 0; o < (1ull << outer.size()); ++o) {
            uint32_t ho = 0;
            for (size_t i = 0; i < outer.size(); ++i) ho |= (uint32_t)((o >> i) & 1u) << outer[i];
            for (int k = 0; k <= ws; ++k) {
                const int m = nup - __builtin_popcount(ho) - k;
                if (m < 0 || m > L) continue;
                const int64_t nchunk = (n_choose_k(L, m) + 7) / 8;
                for (int64_t c = 0; c < nchunk; ++c) items.push_back((uint64_t)ho | ((uint64_t)k << 32) | ((uint64_t)c << 40));
            }
        }
        pl.ws[q] = ws;
        pl.nwb[q] = (int)wb.size();
        pl.nitems_p[q] = (int64_t)items.size();
        auto up = [](auto **dst, const auto &v) -> xd_status {
            using E = typename std::remove_reference<decltype(v)>::type::value_type;
            XD_CUDA(dev_malloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(E)));
            if (!v.empty()) XD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice));
            return XD_OK;
        };
        XD_TRY(up(&pl.d_wlist[q], wlist));
        XD_TRY(up(&pl.d_woff[q], woff));
        XD_TRY(up(&pl.d_wrank[q], wrank));
        XD_TRY(up(&pl.d_wdep[q], wdep));
        XD_TRY(up(&pl.d_wbond[q], wb));
        XD_TRY(up(&pl.d_pitems[q], items));
    }
    // k_main's items: the prefix sites of the cross bonds lowest in the key
    std::vector<int> cl;
    for (size_t c = 0; c < s.h_csite.size(); c += 3) cl.push_back(s.h_csite[c]);
    std::sort(cl.begin(), cl.end());
    cl.erase(std::unique(cl.begin(), cl.end()), cl.end());
    pl.cross_low = cl;
    for (int v = 0; v < 2; ++v) {
        const int KB = v == 0 ? 4 : 8;
        const std::vector<uint32_t> items = ordered_items(P, nup, L, KB, kEmpty, cl);
        pl.nitems[v] = (int64_t)items.size() / KB;
        XD_CUDA(dev_malloc((void **)&pl.d_items[v], std::max<size_t>(1, items.size()) * sizeof(uint32_t)));
        if (!items.empty())
            XD_CUDA(cudaMemcpy(pl.d_items[v], items.data(), items.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    pl.ok = true;
    return XD_OK;
}

void pass_layout_free(xd_basis_s *b) {
    PassLayoutHost &pl = b->pass;
    for (int q = 0; q < 4; ++q) {
        cudaFree(pl.d_wlist[q]);
        cudaFree(pl.d_woff[q]);
        cudaFree(pl.d_wrank[q]);
        cudaFree(pl.d_wdep[q]);
        cudaFree(pl.d_wbond[q]);
        cudaFree(pl.d_pitems[q]);
    }
    for (int v = 0; v < 2; ++v) cudaFree(pl.d_items[v]);
    pl = PassLayoutHost();
}

// The FP64 workspace (8 bytes per row, the two state words and the partials
// of the statistics pass) is allocated on first use.  When it does not fit,
// the call returns XD_ENOMEM and this product takes the FP64 block kernel;
// the next product tries again (the drivers that hold several vectors
// release the workspace when their own vectors do not fit, x64_release).
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
        lanczos_forget(h, false);  // captured Lanczos steps read the workspace
        cudaFree(h->d_x64_x);
        h->d_x64_x = nullptr;
    }
}

// the passes over the prefix blocks, then k_main, for one arithmetic
template <class Pol, int KB>
static xd_status launch_passes(const xd_ham_s *h, const typename Pol::V *x, typename Pol::Y *y, cudaStream_t st) {
    const xd_basis_s *b = h->b;
    const SpmmLayoutHost &s = b->spmm;
    const PassLayoutHost &pl = b->pass;
    const bool fx = Pol::kMode == 1;
    const void *coef = fx ? h->d_x64_fxc : h->d_x64_dfc;
    typename Pol::Acc *acc = (typename Pol::Acc *)y;
    grid_for(1, 1, 1);
    for (int q = 0; q < pl.npass; ++q) {
        TPassParams tp;
        tp.nup = b->nup;
        tp.hi_off = s.d_hi_off;
        tp.lo_off = s.d_lo_off;
        tp.items = pl.d_pitems[q];
        tp.nitems = pl.nitems_p[q];
        tp.wlist = pl.d_wlist[q];
        tp.woff = pl.d_woff[q];
        tp.wrank = pl.d_wrank[q];
        tp.wdep = pl.d_wdep[q];
        tp.wbond = pl.d_wbond[q];
        tp.nwb = pl.nwb[q];
        tp.ws = pl.ws[q];
        tp.coef = coef;
        tp.state = h->d_x64_state;
        const size_t tsm = TPassSmem(tp.ws, tp.nwb, sizeof(typename Pol::V), sizeof(typename Pol::C),
                                     sizeof(typename Pol::Acc), q == 0).total;
        auto tk = q == 0 ? k_tpass<Pol, true> : k_tpass<Pol, false>;
        XD_CUDA(cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm));
        int tper = 0;
        XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tper, tk, kT, tsm));
        if (tper < 1) {
            set_error("U(1) product: %zu bytes of shared memory do not fit", tsm);
            return XD_ERANGE;
        }
        const int tgrid = (int)std::min<int64_t>(std::max<int64_t>(1, tp.nitems), (int64_t)g_num_sms * tper);
        tk<<<tgrid, kT, tsm, st>>>(tp, x, acc);
        XD_CUDA(cudaGetLastError());
    }
    MainParams p;
    p.nup = b->nup;
    p.hi_off = s.d_hi_off;
    p.lo_off = s.d_lo_off;
    p.lo_list = s.d_lo_list;
    p.lo_rank = s.d_lo_rank;
    p.items = pl.d_items[KB == 4 ? 0 : 1];
    p.nitems = pl.nitems[KB == 4 ? 0 : 1];
    p.xtab = s.d_xtab;
    p.pre = s.d_pre;
    p.npre = s.npre;
    p.cross = s.d_cross;
    p.ncross = s.ncross;
    p.csite = s.d_csite;
    p.ncsite = s.ncsite;
    p.post = h->d_x64_post;
    p.npost = s.npost;
    p.coef = coef;
    p.dpost = fx ? h->d_x64_fxp : h->d_x64_dfp;
    p.bdiag = fx ? h->d_x64_fxd : h->d_x64_dfd;
    p.nb = b->nb;
    p.dcross_d = h->x64_dcross_d;
    p.dcross_i = h->x64_dcross_i;
    p.qs = h->x64_qs;
    p.B = h->x64_B;
    p.state = h->d_x64_state;
    const MainSmem<Pol, KB> lay(p);
    auto kern = k_main<Pol, KB>;
    XD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total));
    int per_sm = 0;
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, lay.total));
    if (per_sm < 1) {
        set_error("U(1) product: %zu bytes of shared memory do not fit", lay.total);
        return XD_ERANGE;
    }
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, p.nitems), (int64_t)g_num_sms * per_sm);
    kern<<<grid, kT, lay.total, st>>>(p, x, acc, y);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// the batched layout has L = 12 for every block it is built for (N >= 24)
bool passes_usable(const xd_ham_s *h) {
    const xd_basis_s *b = h->b;
    return b->spmm.ok && b->spmm.L == kL && h->d_x64_tab != nullptr;
}

// Statistics of x, the choice of arithmetic and the conversion on the
// device; both arithmetics' kernels are launched and those not chosen return
// at once (no host synchronisation).
xd_status passes_apply_f64(const xd_ham_s *h, const void *x, void *y, cudaStream_t st) {
    xd_ham_s *hm = const_cast<xd_ham_s *>(h);
    const int64_t dim = h->b->dim;
    XD_TRY(pass_layout_build(h->b));
    XD_TRY(x64_workspace(hm, dim));
    const int g1 = grid_for(dim, kStatThreads, kStatPerSm);
    ExpSum *part = (ExpSum *)((unsigned char *)h->d_x64_state + 16);
    k_x64_stats<<<g1, kStatThreads, 0, st>>>((const unsigned long long *)x, dim, part);
    k_x64_convert<<<g1, kStatThreads, 0, st>>>((const unsigned long long *)x, dim, part, g1, h->x64_fx_ok ? 1 : 0,
                                               h->x64_B, h->d_x64_state, h->d_x64_x);
    XD_CUDA(cudaGetLastError());
    if (h->x64_fx_ok) XD_TRY((launch_passes<PolFX, 4>(h, (const long long *)h->d_x64_x, (double *)y, st)));
    return launch_passes<PolDF, 4>(h, (const float2 *)h->d_x64_x, (double *)y, st);
}

}  // namespace xd

// xd_lanczos.cu -- seeded start vectors, fused vector kernels, the Lanczos
// driver (eigvals_lanczos / eig0 of Sec. 3.6.1) and the host tridiagonal
// eigensolver (a6, a7).
//
// Krylov vectors are kept unnormalised with a host scale sigma_k so that
// v_k = sigma_k u_k; one step is
//     w     = H u_k                                   (xd_apply)
//     w     = sigma_k w - beta_{k-1} sigma_{k-1} u_{k-1},  alpha_k = sigma_k <w, u_k>
//     w     = w - alpha_k sigma_k u_k,                beta_k = ||w||
//     u_{k+1} = w, sigma_{k+1} = 1 / beta_k.
// Complex vectors with real scalars are real vectors of twice the length,
// and alpha = Re <v, Hv> for Hermitian H, so the same kernels serve them.
// Dot products: FP64 fused multiply-adds for double storage; for float
// storage each thread keeps an exact float product split (FMA) and a
// compensated float pair sum (FP64-class), and partial sums meet in FP64.
// All reductions run in a fixed order (per-CTA partials, then one pass).

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cooperative_groups.h>

#include "xd_internal.cuh"
#include "xd_tridiag.h"
#include "xd_u1_rows.cuh"

namespace xd {

namespace {

constexpr int kThreads = 256;

// SplitMix64 output for the state advanced from z by its increment.
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += kGolden;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Seeded standard normals: the seed is mixed into the stream state
// k = splitmix64(seed), entry i takes outputs 2i+1 and 2i+2 of the SplitMix64
// stream from k and maps them to (0,1] uniforms for Box-Muller.
template <typename T>
__global__ void k_random(int64_t n, uint64_t seed, T *__restrict__ out, int stride) {
    const uint64_t k = splitmix64(seed);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = k + 2ull * (uint64_t)i * kGolden;
        const uint64_t a = splitmix64(c);
        const uint64_t b = splitmix64(c + kGolden);
        const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
        const double u2 = ((double)(b >> 11) + 1.0) * 0x1.0p-53;
        const double v = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
        out[i * stride] = (T)v;
        if (stride == 2) out[i * stride + 1] = (T)0;
    }
}

struct AccD {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};

// Exact product split and compensated sum in float pairs.
struct AccF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -p);             // a*b = p + pe exactly
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

template <typename T>
struct AccOf;
template <>
struct AccOf<double> {
    using A = AccD;
};
template <>
struct AccOf<float> {
    using A = AccF;
};

// Vector updates with their roundings spelt out (a product, then one fused
// multiply-add), so that every kernel forming a Lanczos vector -- the first
// pass in any of its forms and the second pass that rebuilds the vectors
// from the recorded alpha and beta -- rounds alike and the second pass
// reproduces the first pass's vectors.
// (mul_rn, fma_rn: xd_u1_rows.cuh)

// block-wide sum of one double per thread into part[blockIdx.x] (fixed order)
__device__ __forceinline__ void block_store(double v, double *__restrict__ part) {
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// w = a w + c z (z may be NULL); part = <w, v> for mode 1, <w, w> (the new
// w with itself) for mode 2, no dot for mode 0.  v never aliases w.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_axpby_dot(int64_t n, T *__restrict__ w, T a,
                                                        const T *__restrict__ z, T c,
                                                        const T *__restrict__ v, int mode,
                                                        double *__restrict__ part) {
    typename AccOf<T>::A acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T t = mul_rn(a, w[i]);
        if (z) t = fma_rn(c, z[i], t);
        w[i] = t;
        if (mode == 1) acc.add(t, v[i]);
        else if (mode == 2) acc.add(t, t);
    }
    if (mode) block_store(acc.get(), part);
}

// psi += c u
template <typename T>
__global__ void k_axpy(int64_t n, T *__restrict__ psi, T c, const T *__restrict__ u) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        psi[i] += c * u[i];
}

// Eight independent vectors stored row-major [rows][8] (column c is vector
// c): w_c = a_c w_c + b_c z_c, then part = <w_c, v_c> (mode 1) or <w_c, w_c>
// (mode 2) per column, in FP64, fixed order (per-CTA partials [grid][8]).
struct Coef8 {
    double a[8], b[8];
};

__global__ void __launch_bounds__(kThreads) k_axpby_dot8(int64_t rows, double *__restrict__ w, Coef8 co,
                                                         const double *__restrict__ z,
                                                         const double *__restrict__ v, int mode,
                                                         double *__restrict__ part) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double t = co.a[c] * w[i * 8 + c];
            if (z) t = fma(co.b[c], z[i * 8 + c], t);
            w[i * 8 + c] = t;
            if (mode == 1) acc[c] = fma(t, v[i * 8 + c], acc[c]);
            else if (mode == 2) acc[c] = fma(t, t, acc[c]);
        }
    }
    if (!mode) return;
    __shared__ double red[kThreads / 32][8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double s = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = s;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q][threadIdx.x];
        part[(size_t)blockIdx.x * 8 + threadIdx.x] = s;
    }
}

// ---------------------------------------- device-resident Lanczos steps
// The first Lanczos pass keeps its scalars on the device.  A step is the
// product w = H u, then k_lz_axpby1: w = sig w + cz up with <w, u>, whose
// last CTA to finish sums the CTA partials in a fixed order and sets alpha,
// then k_lz_axpby2: w = w + ca u with <w, w>, whose last CTA sets beta, the
// stop test and the next step's coefficients.  When beta falls below 1e-13
// max|alpha| (or is zero) or the step budget is spent, `done` is set and
// every later vector kernel returns at once, so the host can replay captured
// steps and look at the flag only every few steps.
struct LzDev {
    double sig;     // 1 / |w| of the current vector (its normalisation)
    double cz;      // -beta_{k-1} sig_{k-1}: coefficient of the previous vector
    double ca;      // -alpha_k sig_k
    double amax;    // max |alpha| so far
    int k;          // steps done
    int done;       // 1 once the run has stopped
    int max_iter;
    unsigned arrived;  // CTAs done with the current vector kernel
};

// The last CTA of a grid to store its partial returns true (and has the
// other CTAs' partials visible); the counter is reset for the next kernel.
__device__ __forceinline__ bool last_cta(LzDev *sd) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&sd->arrived, 1u) == gridDim.x - 1;
        if (last) sd->arrived = 0;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// sum of n CTA partials by one warp: lane l adds entries l, l + 32, ... in
// order, then a fixed shuffle tree (the same order on every call)
__device__ __forceinline__ double warp_sum_parts(const double *part, int n) {
    const int lane = threadIdx.x & 31;
    double d = 0.0;
    for (int i = lane; i < n; i += 32) d += __ldcg(part + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    return d;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_lz_axpby1(int64_t n, T *__restrict__ w, const T *__restrict__ up,
                                                        const T *__restrict__ u, LzDev *sd, double *part,
                                                        double *__restrict__ alpha) {
    if (sd->done) return;
    const T a = (T)sd->sig, c = (T)sd->cz;
    typename AccOf<T>::A acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T t = fma_rn(c, up[i], mul_rn(a, w[i]));
        w[i] = t;
        acc.add(t, u[i]);
    }
    block_store(acc.get(), part);
    if (last_cta(sd) && threadIdx.x < 32) {
        // alpha_k = sig <w, u>
        const double al = sd->sig * warp_sum_parts(part, gridDim.x);
        if (threadIdx.x == 0) {
            alpha[sd->k] = al;
            sd->ca = -al * sd->sig;
            sd->amax = fmax(sd->amax, fabs(al));
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_lz_axpby2(int64_t n, T *__restrict__ w, const T *__restrict__ u,
                                                        LzDev *sd, double *part, double *__restrict__ beta) {
    if (sd->done) return;
    const T c = (T)sd->ca;
    typename AccOf<T>::A acc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T t = fma_rn(c, u[i], w[i]);
        w[i] = t;
        acc.add(t, t);
    }
    block_store(acc.get(), part);
    if (last_cta(sd) && threadIdx.x < 32) {
        // beta_k = |w|; the stop test; the next step's coefficients
        const double bt = sqrt(fmax(warp_sum_parts(part, gridDim.x), 0.0));
        if (threadIdx.x) return;
        beta[sd->k] = bt;
        sd->k += 1;
        if (!(bt > 0.0) || bt < 1e-13 * sd->amax || sd->k >= sd->max_iter) {
            sd->done = 1;
        } else {
            sd->cz = -bt * sd->sig;
            sd->sig = 1.0 / bt;
        }
    }
}

// The whole first pass in one cooperative launch, for small U(1) blocks
// whose product is the plain row loop, one row per thread: the row's state
// word is unranked once and kept in a register.  A step is two phases
// separated by grid-wide barriers:
//   product: w_r = (H u)_r in the row loop's order and roundings
//     (xd_u1_rows.cuh), so that the vectors are those of the second pass bit
//     for bit, with the partial dots <H u, u> and <up, u>, so that
//     alpha_k = sig <sig H u + cz up, u> (the modified form) needs no
//     further pass;
//   update: w = sig w + cz up - alpha_k sig u, with the partial norms.
// Every CTA sums the partials itself in the fixed order of warp_sum_parts,
// so all CTAs hold the same alpha, beta and stop decision; CTA 0 records
// them.  A thread updates only its own row, so only the product's gathers
// read other CTAs' writes (through L2).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_lz_persist(U1View u1, const double *__restrict__ bond, int nb,
                                                         T *b0, T *b1, T *b2, LzDev *sd, double *pa,
                                                         double *pb, double *pc, double *__restrict__ alpha,
                                                         double *__restrict__ beta) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sm_mask = (uint64_t *)smem;
    T *sm_half = (T *)(sm_mask + nb);
    __shared__ uint64_t sh_range[2];
    __shared__ double sh_sum[2];
    u1rows::stage_bonds(bond, nb, sm_mask, sm_half);
    const T jq = (T)bond[2 * nb];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // this thread's row
    const u1rows::RowState rs = u1rows::unrank_tile(u1, (int64_t)blockIdx.x * blockDim.x, r, sh_range);
    double sig = sd->sig, cz = sd->cz, amax = sd->amax;
    int k = sd->k;
    const int max_iter = sd->max_iter;
    const bool rec = blockIdx.x == 0 && threadIdx.x == 0;
    T *up = b0, *u = b1, *w = b2;
    for (;;) {
        double d1 = 0.0, d2 = 0.0;
        if (rs.valid) {
            T acc = T(0), dsub = T(0);
            for (int b = 0; b < nb; ++b) {
                const uint64_t mk = sm_mask[b];
                const uint64_t t = rs.s & mk;
                if (t != 0 && t != mk) {
                    const T cf = sm_half[b];
                    acc = fma_rn(cf, __ldcg(u + u1rows::rank_of(u1, rs.s ^ mk)), acc);
                    dsub += cf;
                }
            }
            const T ur = u[r];
            const T wr = fma_rn(jq - dsub, ur, acc);
            w[r] = wr;
            d1 = (double)wr * (double)ur;
            d2 = (double)up[r] * (double)ur;
        }
        block_store(d1, pa);
        __syncthreads();  // thread 0 has read block_store's scratch before it is reused
        block_store(d2, pb);
        grid.sync();
        if (threadIdx.x < 32) {
            const double s1 = warp_sum_parts(pa, gridDim.x), s2 = warp_sum_parts(pb, gridDim.x);
            if (threadIdx.x == 0) {
                sh_sum[0] = s1;
                sh_sum[1] = s2;
            }
        }
        __syncthreads();
        const double al = sig * (sig * sh_sum[0] + cz * sh_sum[1]);  // alpha_k
        if (rec) alpha[k] = al;
        amax = fmax(amax, fabs(al));
        double d3 = 0.0;
        if (rs.valid) {
            const T t1 = fma_rn((T)cz, up[r], mul_rn((T)sig, w[r]));
            const T t = fma_rn((T)(-al * sig), u[r], t1);
            w[r] = t;
            d3 = (double)t * (double)t;
        }
        block_store(d3, pc);
        grid.sync();
        if (threadIdx.x < 32) {
            const double s3 = warp_sum_parts(pc, gridDim.x);
            if (threadIdx.x == 0) sh_sum[0] = s3;
        }
        __syncthreads();
        const double bt = sqrt(fmax(sh_sum[0], 0.0));  // beta_k = |w|
        if (rec) beta[k] = bt;
        k += 1;
        if (!(bt > 0.0) || bt < 1e-13 * amax || k >= max_iter) break;  // the same in every CTA
        cz = -bt * sig;
        sig = 1.0 / bt;
        T *t = up;
        up = u;
        u = w;
        w = t;
        __syncthreads();  // sh_sum read by every thread before the next step writes it
    }
    if (rec) {
        sd->k = k;
        sd->done = 1;
    }
}

// out[c] = sum over CTAs of part[cta][c], fixed order
__global__ void k_sum8(const double *__restrict__ part, int n, double *__restrict__ out) {
    if (threadIdx.x >= 8 || blockIdx.x) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[(size_t)i * 8 + threadIdx.x];
    out[threadIdx.x] = s;
}

// out += (cr + i ci) u on interleaved complex vectors of n entries
__global__ void k_axpy_c(int64_t n, double2 *__restrict__ out, double cr, double ci,
                         const double2 *__restrict__ u) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = u[i];
        double2 o = out[i];
        o.x += cr * v.x - ci * v.y;
        o.y += cr * v.y + ci * v.x;
        out[i] = o;
    }
}

// *out = sum of n partials (one warp, the fixed order of warp_sum_parts)
__global__ void k_sum(const double *__restrict__ part, int n, double *__restrict__ out) {
    if (blockIdx.x || threadIdx.x >= 32) return;
    const double s = warp_sum_parts(part, n);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace

xd_status vec_random(int64_t n, uint64_t seed, void *out, xd_dtype dt, cudaStream_t st) {
    if (n == 0) return XD_OK;
    int grid = grid_for(n, kThreads, 16);
    if (dt == XD_F32) k_random<float><<<grid, kThreads, 0, st>>>(n, seed, (float *)out, 1);
    else k_random<double><<<grid, kThreads, 0, st>>>(n, seed, (double *)out, dt == XD_C128 ? 2 : 1);
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// ------------------------------------------------------------ host side

static xd_status ensure_lanczos_partials(xd_ham_s *h, int n) {
    if (h->lzpart_n >= n) return XD_OK;
    lanczos_forget(h, false);  // captured steps write into the old partials
    cudaFree(h->d_lzpart);
    h->d_lzpart = nullptr;
    h->lzpart_n = 0;
    XD_CUDA(dev_malloc((void **)&h->d_lzpart, sizeof(double) * n));
    h->lzpart_n = n;
    return XD_OK;
}

struct LzWork {
    void *u_prev, *u, *w;
    double *part, *scal;
    int grid;
};

template <typename T>
static xd_status lz_axpby(int64_t n, T *w, double a, const T *z, double c, const T *v,
                          const LzWork &lw, cudaStream_t st, double *dot) {
    // a dot of w with itself reads the updated w, never through a second pointer
    const int mode = !v ? 0 : (v == w ? 2 : 1);
    k_axpby_dot<T><<<lw.grid, kThreads, 0, st>>>(n, w, (T)a, z, (T)c, mode == 1 ? v : nullptr, mode,
                                                 mode ? lw.part : nullptr);
    XD_CUDA(cudaGetLastError());
    if (dot) {
        k_sum<<<1, 32, 0, st>>>(lw.part, lw.grid, lw.scal);
        XD_CUDA(cudaGetLastError());
        XD_CUDA(cudaMemcpyAsync(dot, lw.scal, sizeof(double), cudaMemcpyDeviceToHost, st));
        XD_CUDA(cudaStreamSynchronize(st));
    }
    return XD_OK;
}

// The first Lanczos pass with its scalars on the device: three steps (one
// turn of the three vectors' roles) are captured in a CUDA graph on a
// stream of the handle's own and replayed; the host reads the state every
// few replays (every replay once the products are costly, so that at most
// two products run after the stop).  A product is run once before the capture so that its
// tables and workspaces exist.  For blocks whose three vectors take at most
// kLzKeep bytes the captured steps and their vectors stay with the handle
// for the next run of the same storage and step budget (dropped when the
// couplings change); larger runs free them at the end.
constexpr int kLzCheckSmall = 8;       // replays between looks at the state, blocks below 2^20 rows
constexpr size_t kLzKeep = 256u << 20;

void lanczos_forget(xd_ham_s *h, bool all) {
    if (h->lz_exec) cudaGraphExecDestroy(h->lz_exec);
    h->lz_exec = nullptr;
    for (int q = 0; q < 3; ++q) {
        cudaFree(h->lz_buf[q]);
        h->lz_buf[q] = nullptr;
    }
    h->lz_key_dt = -1;
    h->lz_key_iter = 0;
    if (!all) return;
    if (h->lz_stream) cudaStreamDestroy(h->lz_stream);
    h->lz_stream = nullptr;
    cudaFree(h->lz_dstate);
    h->lz_dstate = nullptr;
    if (h->lz_hstate) cudaFreeHost(h->lz_hstate);
    h->lz_hstate = nullptr;
    cudaFree(h->lz_ab);
    h->lz_ab = nullptr;
    h->lz_ab_cap = 0;
}

// Launch shape of the cooperative first pass, or false where it does not
// apply: a U(1) block without the block layouts (its product is the plain
// row loop), one row per thread with every CTA resident, a device with
// cooperative launch.
struct LzSmall {
    int grid;
    size_t smem;
};

template <typename T>
static bool lz_small_shape(const xd_ham_s *h, LzSmall *out) {
    const xd_basis_s *b = h->b;
    if (b->sym || b->blk.ok || b->spmm.ok || b->dim > (1 << 22)) return false;
    int dev = 0, coop = 0, per_sm = 0;
    const size_t smem = (size_t)b->nb * (sizeof(uint64_t) + sizeof(T));
    if (smem > 48 * 1024 || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lz_persist<T>, kThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    grid_for(1, 1, 1);
    const int64_t need = (b->dim + kThreads - 1) / kThreads;
    if (need > (int64_t)per_sm * g_num_sms) return false;
    out->grid = (int)need;
    out->smem = smem;
    return true;
}

template <typename T>
static xd_status lanczos_pass1_graph(xd_ham_s *h, int max_iter, uint64_t seed, xd_dtype dt, double *alpha,
                                     double *beta, int *n_iter) {
    const xd_basis_s *b = h->b;
    const int64_t n = b->dim * (b->cplx ? 2 : 1);
    const size_t vbytes = (size_t)n * sizeof(T);
    const bool keep = 3 * vbytes <= kLzKeep;
    LzWork lw;
    lw.grid = grid_for(n, kThreads, 8);
    // small blocks whose product is the plain row loop: one cooperative
    // launch for the whole pass (all its CTAs resident at once)
    LzSmall lzs{0, 0};
    const bool persist = lz_small_shape<T>(h, &lzs);
    const int pstride = std::max(lw.grid, lzs.grid);  // three arrays of partials
    XD_TRY(ensure_lanczos_partials(h, 3 * pstride));
    lw.part = h->d_lzpart;
    lw.scal = h->d_scal;
    double *part1 = h->d_lzpart, *part2 = h->d_lzpart + pstride;
    cudaError_t e = cudaSuccess;
    if (!h->lz_stream) e = cudaStreamCreateWithFlags(&h->lz_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->lz_dstate) e = dev_malloc(&h->lz_dstate, sizeof(LzDev));
    if (e == cudaSuccess && !h->lz_hstate) e = cudaMallocHost(&h->lz_hstate, sizeof(LzDev));
    if (e == cudaSuccess && h->lz_ab_cap < max_iter) {
        cudaFree(h->lz_ab);
        h->lz_ab = nullptr;
        h->lz_ab_cap = 0;
        e = dev_malloc((void **)&h->lz_ab, sizeof(double) * 2 * (size_t)max_iter);
        if (e == cudaSuccess) h->lz_ab_cap = max_iter;
        lanczos_forget(h, false);  // the captured steps write into the old array
    }
    if (e != cudaSuccess) return cuda_status(e, "Lanczos workspace");
    cudaStream_t st = h->lz_stream;
    LzDev *d_sd = (LzDev *)h->lz_dstate, *h_sd = (LzDev *)h->lz_hstate;
    double *d_ab = h->lz_ab;
    const int abcap = h->lz_ab_cap;
    const bool cached = h->lz_exec && h->lz_key_dt == (int)dt && h->lz_key_iter == max_iter;
    if (!cached) lanczos_forget(h, false);
    T *buf[3] = {(T *)h->lz_buf[0], (T *)h->lz_buf[1], (T *)h->lz_buf[2]};
    double *d_abb = h->lz_ab + abcap;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (!buf[k]) e = dev_malloc_vec(h, (void **)&buf[k], std::max<size_t>(vbytes, 16));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = cached ? h->lz_exec : nullptr;
    xd_status rc = e == cudaSuccess ? XD_OK : cuda_status(e, "cudaMalloc(Lanczos vectors)");
    do {
        if (rc != XD_OK) break;
        T *up = buf[0], *u = buf[1], *w = buf[2];
        if ((rc = vec_random(b->dim, seed, u, dt, st)) != XD_OK) break;
        if ((e = cudaMemsetAsync(up, 0, vbytes, st)) != cudaSuccess) {
            rc = cuda_status(e, "cudaMemsetAsync");
            break;
        }
        double nrm2 = 0.0;
        if ((rc = lz_axpby<T>(n, u, 1.0, nullptr, 0.0, u, lw, st, &nrm2)) != XD_OK) break;
        if (!(nrm2 > 0.0)) {
            set_error("Lanczos: zero start vector");
            rc = XD_EINVAL;
            break;
        }
        *h_sd = LzDev{1.0 / sqrt(nrm2), 0.0, 0.0, 0.0, 0, 0, max_iter, 0u};
        if ((e = cudaMemcpyAsync(d_sd, h_sd, sizeof(LzDev), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            rc = cuda_status(e, "Lanczos state");
            break;
        }
        if (persist) {
            // the whole pass in one cooperative launch
            const int nbh = b->nb;
            U1View u1 = b->u1view();
            const double *bond = h->d_bond;
            T *p0 = up, *p1 = u, *p2 = w;
            double *part3 = h->d_lzpart + 2 * pstride;
            void *args[] = {&u1, (void *)&bond, (void *)&nbh, &p0, &p1, &p2, &d_sd, &part1, &part2, &part3, &d_ab,
                            (void *)&d_abb};
            e = cudaLaunchCooperativeKernel((const void *)k_lz_persist<T>, dim3(lzs.grid), dim3(kThreads), args,
                                            lzs.smem, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_sd, d_sd, sizeof(LzDev), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                rc = cuda_status(e, "Lanczos (cooperative)");
                break;
            }
        } else if (!exec) {
            // one product outside the capture (tables, workspaces)
            if ((rc = xd_apply(h, u, w, dt, 1, (xd_stream)st)) != XD_OK) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = cuda_status(e, "Lanczos start");
                break;
            }
            if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
                rc = cuda_status(e, "cudaStreamBeginCapture");
                break;
            }
            xd_status cap = XD_OK;
            T *cu = u, *cup = up, *cw = w;
            for (int j = 0; j < 3 && cap == XD_OK; ++j) {
                cap = xd_apply(h, cu, cw, dt, 1, (xd_stream)st);
                if (cap != XD_OK) break;
                k_lz_axpby1<T><<<lw.grid, kThreads, 0, st>>>(n, cw, cup, cu, d_sd, part1, d_ab);
                k_lz_axpby2<T><<<lw.grid, kThreads, 0, st>>>(n, cw, cu, d_sd, part2, d_ab + abcap);
                T *t = cup;
                cup = cu;
                cu = cw;
                cw = t;
            }
            e = cudaStreamEndCapture(st, &graph);
            if (cap != XD_OK) {
                rc = cap;
                break;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) {
                rc = cuda_status(e, "Lanczos graph");
                break;
            }
        }
        const int every = b->dim < (1 << 20) ? kLzCheckSmall : 1;
        for (int rep = 0; !persist && e == cudaSuccess;) {
            e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) break;
            if (++rep % every == 0 || 3 * rep >= max_iter) {
                e = cudaMemcpyAsync(h_sd, d_sd, sizeof(LzDev), cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e == cudaSuccess && h_sd->done) break;
            }
        }
        if (e != cudaSuccess) {
            rc = cuda_status(e, "Lanczos steps");
            break;
        }
        const int k = h_sd->k;
        std::vector<double> ab(2 * (size_t)abcap);
        e = cudaMemcpy(ab.data(), d_ab, sizeof(double) * ab.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rc = cuda_status(e, "Lanczos coefficients");
            break;
        }
        for (int q = 0; q < k; ++q) {
            alpha[q] = ab[q];
            beta[q] = ab[abcap + q];
        }
        *n_iter = k;
    } while (0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(st);
    if (rc == XD_OK && keep) {
        h->lz_exec = exec;
        for (int q = 0; q < 3; ++q) h->lz_buf[q] = buf[q];
        h->lz_key_dt = (int)dt;
        h->lz_key_iter = max_iter;
    } else {
        if (exec) cudaGraphExecDestroy(exec);
        h->lz_exec = nullptr;
        for (int q = 0; q < 3; ++q) {
            cudaFree(buf[q]);
            h->lz_buf[q] = nullptr;
        }
        h->lz_key_dt = -1;
    }
    return rc;
}

// One Lanczos run.  Without coef it is the first pass (device-resident,
// lanczos_pass1_graph); with coef it is the second pass of eig0 (Sec.
// 3.6.1): the same recurrence from the same start, with the recorded alpha
// and beta, accumulating psi = sum_k coef[k] v_k.
template <typename T>
static xd_status lanczos_run(xd_ham_s *h, int max_iter, uint64_t seed, xd_dtype dt, double *alpha,
                             double *beta, int *n_iter, const double *coef, T *psi) {
    if (!coef) return lanczos_pass1_graph<T>(h, max_iter, seed, dt, alpha, beta, n_iter);
    const xd_basis_s *b = h->b;
    const int64_t n = b->dim * (b->cplx ? 2 : 1);
    cudaStream_t st = 0;
    LzWork lw;
    lw.grid = grid_for(n, kThreads, 8);
    const size_t vbytes = (size_t)n * sizeof(T);
    XD_TRY(ensure_lanczos_partials(h, lw.grid));
    lw.part = h->d_lzpart;
    lw.scal = h->d_scal;
    T *buf[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = dev_malloc_vec(h, (void **)&buf[k], std::max<size_t>(vbytes, 16));
        if (e != cudaSuccess) {
            for (int q = 0; q < k; ++q) cudaFree(buf[q]);
            return cuda_status(e, "cudaMalloc(Lanczos vectors)");
        }
    }
    xd_status rc = XD_OK;
    T *up = buf[0], *u = buf[1], *w = buf[2];
    do {
        if ((rc = vec_random(b->dim, seed, u, dt, st)) != XD_OK) break;
        cudaError_t e0 = cudaMemsetAsync(up, 0, vbytes, st);
        if (e0 != cudaSuccess) {
            rc = cuda_status(e0, "cudaMemsetAsync");
            break;
        }
        double nrm2 = 0.0;
        if ((rc = lz_axpby<T>(n, u, 1.0, nullptr, 0.0, u, lw, st, &nrm2)) != XD_OK) break;
        if (!(nrm2 > 0.0)) {
            set_error("Lanczos: zero start vector");
            rc = XD_EINVAL;
            break;
        }
        double sig = 1.0 / sqrt(nrm2), sig_prev = 0.0, beta_prev = 0.0;
        const int steps = *n_iter;
        for (int k = 0; k < steps; ++k) {
            k_axpy<T><<<lw.grid, kThreads, 0, st>>>(n, psi, (T)(coef[k] * sig), u);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                rc = cuda_status(e, "k_axpy");
                break;
            }
            if (k == steps - 1) break;
            if ((rc = xd_apply(h, u, w, dt, 1, (xd_stream)st)) != XD_OK) break;
            if ((rc = lz_axpby<T>(n, w, sig, up, -beta_prev * sig_prev, nullptr, lw, st, nullptr)) != XD_OK) break;
            if ((rc = lz_axpby<T>(n, w, 1.0, u, -alpha[k] * sig, nullptr, lw, st, nullptr)) != XD_OK) break;
            beta_prev = beta[k];
            sig_prev = sig;
            sig = 1.0 / beta_prev;
            T *t = up;
            up = u;
            u = w;
            w = t;
        }
    } while (0);
    cudaError_t e = cudaStreamSynchronize(st);
    for (int q = 0; q < 3; ++q) cudaFree(buf[q]);
    if (rc == XD_OK && e != cudaSuccess) rc = cuda_status(e, "Lanczos");
    return rc;
}

static xd_status check_lanczos_args(xd_ham h, int max_iter, xd_dtype dt, int nev, double *alpha,
                                    double *beta, int *n_iter, double *evals, double *resid) {
    if (!h || !alpha || !beta || !n_iter || !evals || !resid) {
        set_error("xd_lanczos: NULL argument");
        return XD_EINVAL;
    }
    if (max_iter < 1 || nev < 1) {
        set_error("xd_lanczos: need max_iter >= 1 and nev >= 1");
        return XD_EINVAL;
    }
    const xd_basis_s *b = h->b;
    if (b->dim == 0) {
        set_error("xd_lanczos: empty block");
        return XD_EINVAL;
    }
    if (b->cplx ? dt != XD_C128 : (dt != XD_F64 && (dt != XD_F32 || b->sym))) {
        set_error("xd_lanczos: storage dtype %d not valid for this block", (int)dt);
        return XD_EINVAL;
    }
    return XD_OK;
}

// H on an interleaved complex vector: U(1) blocks (H real) as two real
// right-hand sides, symmetry-adapted blocks through the complex kernel.
static xd_status apply_c(xd_ham_s *h, const double *x, double *y, cudaStream_t st) {
    if (!h->b->sym) return u1_apply(h, x, y, XD_F64, 2, st);
    return sym_apply(h, x, y, XD_C128, st);
}

// exp(-z H) psi0 by the two-pass Lanczos method (Sec. 3.6.2): pass 1 builds
// the tridiagonal T_m from v_1 = psi0 / |psi0| until the error estimate
// |psi0| beta_m |[exp(-z T_m) e_1]_m| drops below tol |psi0|; pass 2 reruns
// the same recurrence (recorded alpha, beta) and sums |psi0| c_k v_k.
static xd_status evolve_run(xd_ham_s *h, const double *psi0, double zr, double zi, int max_iter,
                            double tol, double *out, int *n_iter, double *err) {
    const xd_basis_s *b = h->b;
    const int64_t nc = b->dim, n = 2 * nc;
    cudaStream_t st = 0;
    LzWork lw;
    lw.grid = grid_for(n, kThreads, 8);
    XD_TRY(ensure_lanczos_partials(h, lw.grid));
    lw.part = h->d_lzpart;
    lw.scal = h->d_scal;
    const size_t vbytes = (size_t)n * sizeof(double);
    double *buf[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = dev_malloc_vec(h, (void **)&buf[k], std::max<size_t>(vbytes, 16));
        if (e != cudaSuccess) {
            for (int q = 0; q < k; ++q) cudaFree(buf[q]);
            return cuda_status(e, "cudaMalloc(evolution vectors)");
        }
    }
    std::vector<double> alpha(max_iter), beta(max_iter), cre, cim;
    xd_status rc = XD_OK;
    double nrm0 = 0.0, est = INFINITY;
    int m = 0;
    for (int pass = 0; pass < 2 && rc == XD_OK; ++pass) {
        double *up = buf[0], *u = buf[1], *w = buf[2];
        if (pass == 1) {
            cudaError_t e = cudaMemsetAsync(out, 0, vbytes, st);
            if (e != cudaSuccess) {
                rc = cuda_status(e, "cudaMemsetAsync");
                break;
            }
        }
        cudaError_t e = cudaMemcpyAsync(u, psi0, vbytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(up, 0, vbytes, st);
        if (e != cudaSuccess) {
            rc = cuda_status(e, "evolution start");
            break;
        }
        if (pass == 0) {
            double nrm2 = 0.0;
            if ((rc = lz_axpby<double>(n, u, 1.0, nullptr, 0.0, u, lw, st, &nrm2)) != XD_OK) break;
            nrm0 = sqrt(nrm2);
            if (!(nrm0 > 0.0)) {  // exp(-zH) 0 = 0
                m = 0;
                est = 0.0;
                cudaMemsetAsync(out, 0, vbytes, st);
                break;
            }
        }
        double sig = 1.0 / nrm0, sig_prev = 0.0, beta_prev = 0.0, amax = 0.0;
        const int steps = pass == 0 ? max_iter : m;
        for (int k = 0; k < steps; ++k) {
            if (pass == 1) {
                // out += |psi0| c_k v_k, v_k = sig u
                k_axpy_c<<<lw.grid, kThreads, 0, st>>>(nc, (double2 *)out, nrm0 * cre[k] * sig,
                                                       nrm0 * cim[k] * sig, (const double2 *)u);
                cudaError_t e2 = cudaGetLastError();
                if (e2 != cudaSuccess) {
                    rc = cuda_status(e2, "k_axpy_c");
                    break;
                }
                if (k == steps - 1) break;
                if ((rc = apply_c(h, u, w, st)) != XD_OK) break;
                if ((rc = lz_axpby<double>(n, w, sig, up, -beta_prev * sig_prev, nullptr, lw, st, nullptr)) != XD_OK) break;
                if ((rc = lz_axpby<double>(n, w, 1.0, u, -alpha[k] * sig, nullptr, lw, st, nullptr)) != XD_OK) break;
                beta_prev = beta[k];
            } else {
                if ((rc = apply_c(h, u, w, st)) != XD_OK) break;
                double d1 = 0.0, d2 = 0.0;
                if ((rc = lz_axpby<double>(n, w, sig, up, -beta_prev * sig_prev, u, lw, st, &d1)) != XD_OK) break;
                const double a = sig * d1;
                if ((rc = lz_axpby<double>(n, w, 1.0, u, -a * sig, w, lw, st, &d2)) != XD_OK) break;
                const double bt = sqrt(std::max(d2, 0.0));
                alpha[k] = a;
                beta[k] = bt;
                amax = std::max(amax, fabs(a));
                beta_prev = bt;
                m = k + 1;
                const bool exact = bt < 1e-13 * amax;
                if (exact || k == steps - 1 || (k + 1) % 4 == 0) {
                    expm_tridiag_e1(m, alpha.data(), beta.data(), zr, zi, cre, cim);
                    est = exact ? 0.0 : nrm0 * bt * hypot(cre[m - 1], cim[m - 1]);
                    if (est <= tol * nrm0 || exact) break;
                }
            }
            sig_prev = sig;
            sig = 1.0 / beta_prev;
            double *tmp = up;
            up = u;
            u = w;
            w = tmp;
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    for (int q = 0; q < 3; ++q) cudaFree(buf[q]);
    if (rc == XD_OK && e != cudaSuccess) rc = cuda_status(e, "time evolution");
    if (rc == XD_OK) {
        *n_iter = m;
        *err = est;
    }
    return rc;
}

// w_c = a_c w_c + b_c z_c on eight columns; with want != 0 the per-column
// dots (mode 1 with v, mode 2 with itself) land in host dots[8].
static xd_status axpby8(int64_t rows, double *w, const Coef8 &co, const double *z, const double *v, int mode,
                        const LzWork &lw, cudaStream_t st, double *dots) {
    k_axpby_dot8<<<lw.grid, kThreads, 0, st>>>(rows, w, co, z, v, mode, lw.part);
    XD_CUDA(cudaGetLastError());
    if (mode) {
        k_sum8<<<1, 32, 0, st>>>(lw.part, lw.grid, lw.scal);
        XD_CUDA(cudaGetLastError());
        XD_CUDA(cudaMemcpyAsync(dots, lw.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
        XD_CUDA(cudaStreamSynchronize(st));
    }
    return XD_OK;
}

// Finite-temperature Lanczos: R seeded random starts (start r is the
// standard-normal vector of seed + r), eight at a time through the 8-wide
// product, M plain Lanczos steps each (a column whose beta falls below
// 1e-13 max|alpha| stops there).  alpha, beta: host [R][M]; n_iter: [R].
static xd_status ftlm_run(xd_ham_s *h, int R, int M, uint64_t seed, double *alpha, double *beta, int *n_iter) {
    const xd_basis_s *b = h->b;
    const int64_t rows = b->dim, n = rows * 8;
    cudaStream_t st = 0;
    LzWork lw;
    lw.grid = grid_for(rows, kThreads, 8);
    XD_TRY(ensure_lanczos_partials(h, lw.grid * 8));
    lw.part = h->d_lzpart;
    lw.scal = h->d_scal;
    const size_t vbytes = (size_t)n * sizeof(double);
    double *buf[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = dev_malloc_vec(h, (void **)&buf[k], std::max<size_t>(vbytes, 16));
        if (e != cudaSuccess) {
            for (int q = 0; q < k; ++q) cudaFree(buf[q]);
            return cuda_status(e, "cudaMalloc(FTLM vectors)");
        }
    }
    xd_status rc = XD_OK;
    for (int r0 = 0; r0 < R && rc == XD_OK; r0 += 8) {
        double *up = buf[0], *u = buf[1], *w = buf[2];
        for (int c = 0; c < 8; ++c) {
            k_random<double><<<lw.grid, kThreads, 0, st>>>(rows, seed + (uint64_t)(r0 + c), u + c, 8);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(up, 0, vbytes, st);
        if (e != cudaSuccess) {
            rc = cuda_status(e, "FTLM start");
            break;
        }
        Coef8 one{};
        for (int c = 0; c < 8; ++c) one.a[c] = 1.0;
        double d[8], sig[8], sigp[8], bp[8], amax[8];
        bool live[8];
        if ((rc = axpby8(rows, u, one, nullptr, nullptr, 2, lw, st, d)) != XD_OK) break;
        for (int c = 0; c < 8; ++c) {
            sig[c] = d[c] > 0.0 ? 1.0 / sqrt(d[c]) : 0.0;
            sigp[c] = bp[c] = amax[c] = 0.0;
            live[c] = d[c] > 0.0;
            if (r0 + c < R) n_iter[r0 + c] = 0;
        }
        for (int k = 0; k < M && rc == XD_OK; ++k) {
            if ((rc = u1_apply(h, u, w, XD_F64, 8, st)) != XD_OK) break;
            Coef8 c1{}, c2{};
            for (int c = 0; c < 8; ++c) {
                c1.a[c] = sig[c];
                c1.b[c] = -bp[c] * sigp[c];
            }
            if ((rc = axpby8(rows, w, c1, up, u, 1, lw, st, d)) != XD_OK) break;
            double a[8];
            for (int c = 0; c < 8; ++c) {
                a[c] = sig[c] * d[c];
                c2.a[c] = 1.0;
                c2.b[c] = -a[c] * sig[c];
            }
            if ((rc = axpby8(rows, w, c2, u, nullptr, 2, lw, st, d)) != XD_OK) break;
            for (int c = 0; c < 8; ++c) {
                const double bt = sqrt(std::max(d[c], 0.0));
                if (live[c] && r0 + c < R) {
                    alpha[(size_t)(r0 + c) * M + k] = a[c];
                    beta[(size_t)(r0 + c) * M + k] = bt;
                    n_iter[r0 + c] = k + 1;
                    amax[c] = std::max(amax[c], fabs(a[c]));
                    if (bt < 1e-13 * amax[c]) live[c] = false;
                }
                sigp[c] = sig[c];
                bp[c] = bt;
                sig[c] = live[c] && bt > 0.0 ? 1.0 / bt : 0.0;
                if (!live[c]) bp[c] = 0.0;
            }
            double *tmp = up;
            up = u;
            u = w;
            w = tmp;
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    for (int q = 0; q < 3; ++q) cudaFree(buf[q]);
    if (rc == XD_OK && e != cudaSuccess) rc = cuda_status(e, "FTLM");
    return rc;
}

}  // namespace xd

using namespace xd;

extern "C" {

xd_status xd_ftlm(xd_ham h, int R, int M, uint64_t seed, double *alpha, double *beta, int *n_iter) {
    if (!h || !alpha || !beta || !n_iter) {
        set_error("xd_ftlm: NULL argument");
        return XD_EINVAL;
    }
    if (R < 1 || R > (1 << 16) || M < 1 || M > 2000) {
        set_error("xd_ftlm: R = %d or M = %d out of range", R, M);
        return XD_EINVAL;
    }
    for (size_t q = 0; q < (size_t)R * M; ++q) alpha[q] = beta[q] = 0.0;
    if (h->b->sym) {
        // symmetry-adapted blocks: one Lanczos pass per start on the block's
        // own product (complex vectors on complex blocks), same seeded starts
        const xd_dtype dt = h->b->cplx ? XD_C128 : XD_F64;
        for (int r = 0; r < R; ++r) {
            int n = 0;
            XD_TRY(lanczos_run<double>(h, M, seed + (uint64_t)r, dt, alpha + (size_t)r * M, beta + (size_t)r * M, &n,
                                       nullptr, nullptr));
            n_iter[r] = n;
        }
        return XD_OK;
    }
    return ftlm_run(h, R, M, seed, alpha, beta, n_iter);
}

xd_status xd_ftlm_thermo(int R, int M, const double *alpha, const double *beta, const int *n_iter, double dim,
                         int nT, const double *temps, double *Z, double *E, double *C) {
    if (!alpha || !beta || !n_iter || !temps || !Z || !E || !C || R < 1 || M < 1 || nT < 0) {
        set_error("xd_ftlm_thermo: bad argument");
        return XD_EINVAL;
    }
    // eigenpairs of every tridiagonal; weights |Q_0j|^2
    std::vector<std::vector<double>> ev(R), wt(R);
    double shift = INFINITY;
    for (int r = 0; r < R; ++r) {
        const int m = std::min(std::max(n_iter[r], 0), M);
        std::vector<double> A((size_t)m * m, 0.0), Q;
        for (int k = 0; k < m; ++k) {
            A[(size_t)k * m + k] = alpha[(size_t)r * M + k];
            if (k + 1 < m) A[(size_t)k * m + k + 1] = A[(size_t)(k + 1) * m + k] = beta[(size_t)r * M + k];
        }
        jacobi_eig(m, A, Q, ev[r]);
        wt[r].resize(m);
        for (int j = 0; j < m; ++j) {
            wt[r][j] = Q[j] * Q[j];
            shift = std::min(shift, ev[r][j]);
        }
    }
    for (int q = 0; q < nT; ++q) {
        const double T = temps[q];
        if (!(T > 0.0)) {
            set_error("xd_ftlm_thermo: temperature %d is not positive", q);
            return XD_EINVAL;
        }
        double z = 0.0, e1 = 0.0, e2 = 0.0;
        for (int r = 0; r < R; ++r)
            for (size_t j = 0; j < ev[r].size(); ++j) {
                const double p = wt[r][j] * exp(-(ev[r][j] - shift) / T);
                z += p;
                e1 += ev[r][j] * p;
                e2 += ev[r][j] * ev[r][j] * p;
            }
        E[q] = e1 / z;
        C[q] = (e2 / z - E[q] * E[q]) / (T * T);
        Z[q] = dim / R * z * exp(-shift / T);
    }
    return XD_OK;
}

xd_status xd_evolve(xd_ham h, const void *psi0, double z_re, double z_im, int max_iter, double tol,
                    void *out, int *n_iter, double *err) {
    if (!h || !psi0 || !out || !n_iter || !err) {
        set_error("xd_evolve: NULL argument");
        return XD_EINVAL;
    }
    if (psi0 == out) {
        set_error("xd_evolve: psi0 and out must be distinct");
        return XD_EINVAL;
    }
    if (max_iter < 1 || max_iter > 1000) {
        set_error("xd_evolve: max_iter = %d outside 1..1000", max_iter);
        return XD_EINVAL;
    }
    if (!std::isfinite(z_re) || !std::isfinite(z_im) || !(tol >= 0.0)) {
        set_error("xd_evolve: z and tol must be finite, tol >= 0");
        return XD_EINVAL;
    }
    return evolve_run(h, (const double *)psi0, z_re, z_im, max_iter, tol, (double *)out, n_iter, err);
}

xd_status xd_lanczos_eigenvalues(xd_ham h, int max_iter, uint64_t seed, xd_dtype dt, int nev,
                                 double *alpha, double *beta, int *n_iter, double *evals,
                                 double *resid) {
    XD_TRY(check_lanczos_args(h, max_iter, dt, nev, alpha, beta, n_iter, evals, resid));
    xd_status s = (dt == XD_F32)
                      ? lanczos_run<float>(h, max_iter, seed, dt, alpha, beta, n_iter, nullptr, nullptr)
                      : lanczos_run<double>(h, max_iter, seed, dt, alpha, beta, n_iter, nullptr, nullptr);
    if (s != XD_OK) return s;
    ritz(*n_iter, alpha, beta, nev, evals, resid, nullptr);
    return XD_OK;
}

xd_status xd_lanczos_ground_state(xd_ham h, int max_iter, uint64_t seed, xd_dtype dt, int nev,
                                  double *alpha, double *beta, int *n_iter, double *evals,
                                  double *resid, void *psi0) {
    XD_TRY(check_lanczos_args(h, max_iter, dt, nev, alpha, beta, n_iter, evals, resid));
    if (!psi0) {
        set_error("xd_lanczos_ground_state: psi0 is NULL");
        return XD_EINVAL;
    }
    XD_TRY(xd_lanczos_eigenvalues(h, max_iter, seed, dt, nev, alpha, beta, n_iter, evals, resid));
    std::vector<double> c;
    ritz(*n_iter, alpha, beta, 1, evals, resid, &c);
    const xd_basis_s *b = h->b;
    const int64_t n = b->dim * (b->cplx ? 2 : 1);
    const size_t vbytes = (size_t)n * (dt == XD_F32 ? 4 : 8);
    XD_CUDA(cudaMemset(psi0, 0, vbytes));
    xd_status s = (dt == XD_F32)
                      ? lanczos_run<float>(h, max_iter, seed, dt, alpha, beta, n_iter, c.data(), (float *)psi0)
                      : lanczos_run<double>(h, max_iter, seed, dt, alpha, beta, n_iter, c.data(), (double *)psi0);
    if (s != XD_OK) return s;
    // normalise
    LzWork lw;
    lw.grid = grid_for(n, kThreads, 8);
    XD_TRY(ensure_lanczos_partials(h, lw.grid));
    lw.part = h->d_lzpart;
    lw.scal = h->d_scal;
    double nrm2 = 0.0;
    if (dt == XD_F32) {
        XD_TRY(lz_axpby<float>(n, (float *)psi0, 1.0, nullptr, 0.0, (float *)psi0, lw, 0, &nrm2));
        XD_TRY(lz_axpby<float>(n, (float *)psi0, 1.0 / sqrt(nrm2), nullptr, 0.0, nullptr, lw, 0, nullptr));
    } else {
        XD_TRY(lz_axpby<double>(n, (double *)psi0, 1.0, nullptr, 0.0, (double *)psi0, lw, 0, &nrm2));
        XD_TRY(lz_axpby<double>(n, (double *)psi0, 1.0 / sqrt(nrm2), nullptr, 0.0, nullptr, lw, 0, nullptr));
    }
    XD_CUDA(cudaDeviceSynchronize());
    return XD_OK;
}

xd_status xd_energy_grad(xd_ham h, const void *psi0, xd_dtype dt, double *dEdJ) {
    if (!h || !psi0 || !dEdJ) {
        set_error("xd_energy_grad: NULL argument");
        return XD_EINVAL;
    }
    const int nb = h->b->nb;
    double *d_out = nullptr;
    XD_CUDA(dev_malloc((void **)&d_out, sizeof(double) * nb));
    xd_status s = xd_apply_bilinear(h, psi0, psi0, dt, d_out, nullptr);
    if (s == XD_OK) {
        cudaError_t e = cudaMemcpy(dEdJ, d_out, sizeof(double) * nb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = cuda_status(e, "xd_energy_grad copy");
    }
    cudaFree(d_out);
    return s;
}

}  // extern "C"

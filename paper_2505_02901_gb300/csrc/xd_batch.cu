// xd_batch.cu -- many independent U(1) products in one persistent launch
// (the multi-vector apply of Sec. 5.1 over a batch of blocks; a9).
//
// Work list: instance k owns ceil(dim_k / tile) row tiles; tile t of the
// whole batch maps to (instance, first row) through the prefix sums
// tile0[k].  A persistent grid walks the tiles; a CTA stages the bond table
// of the instance it is working on in shared memory and reuses it while
// consecutive tiles belong to the same instance.  One index computation
// (unrank, flip test, two-table rank) serves all nvec right-hand sides of a
// row, read and written as one contiguous [nvec] record.
//
// Schedule: the threads per CTA and the rows per tile are chosen by a small
// autotuner that takes the median of five timings of every candidate (CUDA
// events) the first time a batch is seen; the chosen launch is captured in a
// CUDA graph and replayed while the batch (handles, vectors, dtype, nvec,
// stream) is unchanged.
//
// Eight FP32 right-hand sides with operators large enough for the prefix
// block layout (N >= 24): one persistent launch of k_batch8 does the whole
// batch.  Its work list is every prefix block of the large operators (the
// eight-vector product of xd_u1_spmm8.cu, one block per unit, largest
// operators first) followed by the row tiles of the small ones; a CTA takes
// the next unit from a counter in device memory, which the last CTA to
// finish resets for the next launch.

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "xd_internal.cuh"
#include "xd_spmm8.cuh"

namespace xd {

namespace {

struct Inst {
    U1View u;
    const double *bond;  // [J | masks | sum J / 4]
    int nb;
    const void *x;
    void *y;
    int64_t tile0;       // first global tile of this instance
};

constexpr int kMaxBatchBonds = 512;

__device__ __forceinline__ uint64_t find_block(const int64_t *__restrict__ hi_off, uint64_t lo,
                                               uint64_t hi, int64_t r) {
    while (lo < hi) {
        uint64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(hi_off + mid) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Rows [row0, row1) of instance I (bond table staged in sm_mask / sm_half).
template <typename T, int NV>
__device__ __forceinline__ void batch_rows(const Inst &I, const uint64_t *sm_mask, const T *sm_half,
                                           uint64_t *sh_range, int64_t row0, int64_t row1) {
    const U1View &u = I.u;
    if (threadIdx.x == 0) {
        uint64_t nh = 1ull << u.P;
        uint64_t h0 = find_block(u.hi_off, 0, nh - 1, row0);
        sh_range[0] = h0;
        sh_range[1] = find_block(u.hi_off, h0, nh - 1, row1 - 1);
    }
    __syncthreads();
    const T jq = (T)I.bond[2 * I.nb];
    const T *__restrict__ x = (const T *)I.x;
    T *__restrict__ y = (T *)I.y;
    for (int64_t r = row0 + threadIdx.x; r < row1; r += blockDim.x) {
        const uint64_t h = find_block(u.hi_off, sh_range[0], sh_range[1], r);
        const int m = u.nup - __popcll(h);
        const uint32_t l = __ldg(u.lo_list + __ldg(u.lo_off + m) + (uint32_t)(r - __ldg(u.hi_off + h)));
        const uint64_t s = (h << u.L) | l;
        T acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = T(0);
        T dsub = T(0);
        for (int b = 0; b < I.nb; ++b) {
            const uint64_t mk = sm_mask[b];
            const uint64_t tt = s & mk;
            if (tt != 0 && tt != mk) {
                const uint64_t f = s ^ mk;
                const int64_t c = __ldg(u.hi_off + (f >> u.L)) + (int64_t)__ldg(u.lo_rank + (f & u.lomask));
                const T cf = sm_half[b];
#pragma unroll
                for (int q = 0; q < NV; ++q) acc[q] += cf * __ldg(x + c * NV + q);
                dsub += cf;
            }
        }
        const T d = jq - dsub;
#pragma unroll
        for (int q = 0; q < NV; ++q) y[r * NV + q] = d * __ldg(x + r * NV + q) + acc[q];
    }
}

// Stages the bond table of instance I.
template <typename T>
__device__ __forceinline__ void batch_stage(const Inst &I, uint64_t *sm_mask, T *sm_half) {
    const uint64_t *masks = (const uint64_t *)(I.bond + I.nb);
    for (int b = threadIdx.x; b < I.nb; b += blockDim.x) {
        sm_mask[b] = masks[b];
        sm_half[b] = (T)(0.5 * I.bond[b]);
    }
}

// Instance of global tile t: the last with tile0 <= t.
__device__ __forceinline__ int batch_find(const Inst *__restrict__ inst, int ninst, int64_t t) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (inst[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T, int NV>
__global__ void k_batch(const Inst *__restrict__ inst, int ninst, int64_t ntiles, int tile_rows) {
    __shared__ uint64_t sm_mask[kMaxBatchBonds];
    __shared__ T sm_half[kMaxBatchBonds];
    __shared__ int sh_k;
    __shared__ uint64_t sh_range[2];
    int cur = -1;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (threadIdx.x == 0) sh_k = batch_find(inst, ninst, t);
        __syncthreads();
        const int k = sh_k;
        const Inst &I = inst[k];
        if (k != cur) {
            batch_stage(I, sm_mask, sm_half);
            cur = k;
        }
        const int64_t row0 = (t - I.tile0) * tile_rows;
        batch_rows<T, NV>(I, sm_mask, sm_half, sh_range, row0, min(row0 + (int64_t)tile_rows, I.u.dim));
        __syncthreads();
    }
}

// One large operator of the fused launch.
struct Big8 {
    sp8::Sp8Params p;
    const float *x;
    float *y;
    int L;
    int64_t unit0;  // its first work unit
};

// Arguments of the fused launch; the large operators' parameters sit in the
// kernel's parameter space, so that their fields are constant-bank operands.
constexpr int kMaxBig8 = 96;

struct Batch8Args {
    int nbig, ninst, tile_rows;
    int64_t ubig, ntiles;
    const Inst *inst;
    unsigned long long *ctr;
    Big8 big[kMaxBig8];
};

// FP32, eight right-hand sides: the prefix blocks of the large operators
// (units [0, ubig)) and the row tiles of the small ones (units [ubig,
// ubig + ntiles)), one unit at a time from ctr[0]; ctr[1] counts the CTAs
// that are done.
__global__ void __launch_bounds__(sp8::kT8, 2) k_batch8(const __grid_constant__ Batch8Args a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int sh_k;
    __shared__ long long sh_t;
    __shared__ uint64_t sm_mask[kMaxBatchBonds];
    __shared__ float sm_half[kMaxBatchBonds];
    __shared__ uint64_t sh_range[2];
    int cur_big = -1, cur_small = -1;
    const int64_t total = a.ubig + a.ntiles;
    for (;;) {
        if (threadIdx.x == 0) sh_t = (long long)atomicAdd(a.ctr, 1ull);
        __syncthreads();
        const int64_t t = sh_t;
        if (t >= total) break;
        if (t < a.ubig) {
            int q = 0;  // last operator with unit0 <= t (the same in every thread)
            {
                int hi = a.nbig - 1;
                while (q < hi) {
                    int mid = (q + hi + 1) >> 1;
                    if (a.big[mid].unit0 <= t) q = mid; else hi = mid - 1;
                }
            }
            const Big8 &B = a.big[q];
            if (q != cur_big) {  // block() starts with a barrier, after which the tables are seen
                switch (B.L) {
                    case 12: sp8::tables<12>(B.p, smem); break;
                    case 11: sp8::tables<11>(B.p, smem); break;
                    default: sp8::tables<10>(B.p, smem);
                }
                cur_big = q;
            }
            const uint32_t h = __ldg(B.p.items + (t - B.unit0));
            if (h != sp8::kEmpty8) {
                switch (B.L) {
                    case 12: sp8::block<12>(B.p, smem, h, B.x, B.y); break;
                    case 11: sp8::block<11>(B.p, smem, h, B.x, B.y); break;
                    default: sp8::block<10>(B.p, smem, h, B.x, B.y);
                }
            }
        } else {
            const int64_t tt = t - a.ubig;
            if (threadIdx.x == 0) sh_k = batch_find(a.inst, a.ninst, tt);
            __syncthreads();
            const int k = sh_k;
            const Inst &I = a.inst[k];
            if (k != cur_small) {
                batch_stage(I, sm_mask, sm_half);
                cur_small = k;
            }
            const int64_t row0 = (tt - I.tile0) * a.tile_rows;
            batch_rows<float, 8>(I, sm_mask, sm_half, sh_range, row0, min(row0 + (int64_t)a.tile_rows, I.u.dim));
        }
        __syncthreads();  // unit done: shared state may be overwritten
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.ctr + 1, 1ull) == (unsigned long long)gridDim.x - 1) {
            a.ctr[0] = 0;  // every CTA has taken its last unit
            a.ctr[1] = 0;
            __threadfence();
        }
    }
}

struct Plan {
    std::vector<const xd_ham_s *> hs;
    std::vector<const void *> xs;
    std::vector<void *> ys;
    std::vector<int> rest, big;  // small instances (row tiles) / large ones (prefix blocks, k_batch8)
    xd_dtype dt;
    int nvec;
    cudaStream_t st;
    Inst *d_inst = nullptr;
    int64_t ntiles = 0;
    int threads = 256, tile_rows = 1024, grid = 1;
    // fused launch (big non-empty)
    std::vector<Big8> hbig;
    int64_t ubig = 0;
    unsigned long long *d_ctr = nullptr;
    size_t smem8 = 0;
    int per_sm8 = 1;
    cudaGraphExec_t exec = nullptr;
    bool tuned = false;
};

void free_plan(Plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    cudaFree(p->d_inst);
    cudaFree(p->d_ctr);
    delete p;
}

std::mutex g_mu;
std::vector<Plan *> g_plans;

template <typename T, int NV>
void launch(const Plan &p, cudaStream_t st) {
    k_batch<T, NV><<<p.grid, p.threads, 0, st>>>(p.d_inst, (int)p.rest.size(), p.ntiles, p.tile_rows);
}

xd_status launch_any(const Plan &p, cudaStream_t st) {
    if (!p.big.empty()) {
        Batch8Args a;
        a.nbig = (int)p.hbig.size();
        a.ninst = (int)p.rest.size();
        a.tile_rows = p.tile_rows;
        a.ubig = p.ubig;
        a.ntiles = p.ntiles;
        a.inst = p.d_inst;
        a.ctr = p.d_ctr;
        std::copy(p.hbig.begin(), p.hbig.end(), a.big);
        k_batch8<<<p.grid, sp8::kT8, p.smem8, st>>>(a);
    } else if (p.dt == XD_F64) {
        switch (p.nvec) {
            case 1: launch<double, 1>(p, st); break;
            case 2: launch<double, 2>(p, st); break;
            case 4: launch<double, 4>(p, st); break;
            default: launch<double, 8>(p, st);
        }
    } else {
        switch (p.nvec) {
            case 1: launch<float, 1>(p, st); break;
            case 2: launch<float, 2>(p, st); break;
            case 4: launch<float, 4>(p, st); break;
            default: launch<float, 8>(p, st);
        }
    }
    XD_CUDA(cudaGetLastError());
    return XD_OK;
}

// Row tiles of the small instances for the current tile_rows; the grid.
xd_status build_table(Plan *p) {
    std::vector<Inst> h(p->rest.size());
    int64_t tiles = 0;
    for (size_t q = 0; q < p->rest.size(); ++q) {
        const int k = p->rest[q];
        const xd_ham_s *hm = p->hs[k];
        h[q].u = hm->b->u1view();
        h[q].bond = hm->d_bond;
        h[q].nb = hm->b->nb;
        h[q].x = p->xs[k];
        h[q].y = p->ys[k];
        h[q].tile0 = tiles;
        tiles += (hm->b->dim + p->tile_rows - 1) / p->tile_rows;
    }
    p->ntiles = tiles;
    const int64_t units = p->ubig + tiles;
    const int64_t resident = p->big.empty() ? (int64_t)g_num_sms * (2048 / p->threads) : (int64_t)g_num_sms * p->per_sm8;
    p->grid = (int)std::max<int64_t>(1, std::min<int64_t>(units, resident));
    if (h.empty()) return XD_OK;
    if (!p->d_inst) XD_CUDA(dev_malloc((void **)&p->d_inst, sizeof(Inst) * h.size()));
    XD_CUDA(cudaMemcpy(p->d_inst, h.data(), sizeof(Inst) * h.size(), cudaMemcpyHostToDevice));
    return XD_OK;
}

// Work units of the large operators (largest first), the unit counter and
// the fused kernel's shared memory.
xd_status build_big(Plan *p) {
    std::stable_sort(p->big.begin(), p->big.end(),
                     [&](int a, int b) { return p->hs[a]->b->dim > p->hs[b]->b->dim; });
    std::vector<Big8> h(p->big.size());
    int64_t units = 0;
    size_t smem = 0;
    for (size_t q = 0; q < p->big.size(); ++q) {
        const int k = p->big[q];
        sp8_params(p->hs[k], &h[q].p);
        h[q].x = (const float *)p->xs[k];
        h[q].y = (float *)p->ys[k];
        h[q].L = p->hs[k]->b->spmm.L;
        if (h[q].L < 10 || h[q].L > 12) {
            set_error("batched product: postfix length %d not supported", h[q].L);
            return XD_ERANGE;
        }
        h[q].unit0 = units;
        units += h[q].p.nprefix;
        const int mb = h[q].L == 12 ? sp8::Sp8Geo<12>::maxblk : h[q].L == 11 ? sp8::Sp8Geo<11>::maxblk
                                                                              : sp8::Sp8Geo<10>::maxblk;
        smem = std::max(smem, sp8::Sp8Smem(h[q].p, mb).total);
    }
    p->ubig = units;
    p->smem8 = smem;
    XD_CUDA(cudaFuncSetAttribute(k_batch8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    XD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->per_sm8, k_batch8, sp8::kT8, smem));
    if (p->per_sm8 < 1) {
        set_error("batched product: %zu bytes of shared memory do not fit", smem);
        return XD_ERANGE;
    }
    p->hbig = h;
    XD_CUDA(dev_malloc((void **)&p->d_ctr, 2 * sizeof(unsigned long long)));
    XD_CUDA(cudaMemset(p->d_ctr, 0, 2 * sizeof(unsigned long long)));
    return XD_OK;
}

// Time each (threads, rows per tile) candidate kTuneReps times after one
// warm launch and keep the one with the smallest median.  The fused launch
// has 512 threads; only its rows per tile are tuned.
constexpr int kTuneReps = 5;

xd_status autotune(Plan *p) {
    if (!p->big.empty()) XD_TRY(build_big(p));
    if (p->rest.empty()) {
        XD_TRY(build_table(p));
        p->tuned = true;
        return XD_OK;
    }
    std::vector<int> cand_threads = {128, 256, 512};
    if (!p->big.empty()) cand_threads = {sp8::kT8};
    const int cand_rows_per_thread[] = {1, 4, 16};
    struct Events {  // destroyed on every return path
        cudaEvent_t e[kTuneReps + 1] = {};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (cudaEvent_t &x : ev.e) XD_CUDA(cudaEventCreate(&x));
    float best = 1e30f;
    int bt = cand_threads[0], br = cand_threads[0];
    for (int th : cand_threads)
        for (int rpt : cand_rows_per_thread) {
            p->threads = th;
            p->tile_rows = th * rpt;
            XD_TRY(build_table(p));
            XD_TRY(launch_any(*p, p->st));  // warm
            XD_CUDA(cudaEventRecord(ev.e[0], p->st));
            for (int r = 0; r < kTuneReps; ++r) {
                XD_TRY(launch_any(*p, p->st));
                XD_CUDA(cudaEventRecord(ev.e[r + 1], p->st));
            }
            XD_CUDA(cudaEventSynchronize(ev.e[kTuneReps]));
            float ms[kTuneReps];
            for (int r = 0; r < kTuneReps; ++r) XD_CUDA(cudaEventElapsedTime(&ms[r], ev.e[r], ev.e[r + 1]));
            std::sort(ms, ms + kTuneReps);
            const float med = ms[kTuneReps / 2];
            if (med < best) {
                best = med;
                bt = th;
                br = th * rpt;
            }
        }
    p->threads = bt;
    p->tile_rows = br;
    XD_TRY(build_table(p));
    p->tuned = true;
    return XD_OK;
}

xd_status capture(Plan *p) {
    cudaStream_t cs;
    XD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const xd_status s = launch_any(*p, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (s != XD_OK && e == cudaSuccess) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_status(e, "batched graph capture");
    return XD_OK;
}

}  // namespace

void batch_forget(const xd_ham_s *h) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        Plan *p = *it;
        if (std::find(p->hs.begin(), p->hs.end(), h) != p->hs.end()) {
            free_plan(p);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace xd

using namespace xd;

extern "C" xd_status xd_batch_apply(int ninst, const xd_ham *hs, const void *const *xs,
                                    void *const *ys, xd_dtype dt, int nvec, xd_stream stream) {
    if (ninst < 1 || !hs || !xs || !ys) {
        set_error("xd_batch_apply: need ninst >= 1 and non-NULL arrays");
        return XD_EINVAL;
    }
    if (dt != XD_F64 && dt != XD_F32) {
        set_error("xd_batch_apply: dtype must be XD_F64 or XD_F32");
        return XD_EINVAL;
    }
    if (nvec != 1 && nvec != 2 && nvec != 4 && nvec != 8) {
        set_error("xd_batch_apply: nvec = %d not in {1, 2, 4, 8}", nvec);
        return XD_EINVAL;
    }
    for (int k = 0; k < ninst; ++k) {
        if (!hs[k] || !xs[k] || !ys[k] || xs[k] == ys[k]) {
            set_error("xd_batch_apply: instance %d has a NULL handle/vector or x == y", k);
            return XD_EINVAL;
        }
        if (hs[k]->b->sym) {
            set_error("xd_batch_apply: instance %d is a symmetric block (U(1) blocks only)", k);
            return XD_EINVAL;
        }
        if (hs[k]->b->nb > kMaxBatchBonds) {
            set_error("xd_batch_apply: instance %d has %d > %d bonds", k, hs[k]->b->nb, kMaxBatchBonds);
            return XD_ERANGE;
        }
    }
    grid_for(1, 1, 1);  // make sure the SM count is known
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    Plan *plan = nullptr;
    for (Plan *p : g_plans) {
        if (p->dt != dt || p->nvec != nvec || p->st != st || (int)p->hs.size() != ninst) continue;
        bool same = true;
        for (int k = 0; k < ninst && same; ++k)
            same = p->hs[k] == hs[k] && p->xs[k] == xs[k] && p->ys[k] == ys[k];
        if (same) {
            plan = p;
            break;
        }
    }
    if (!plan) {
        plan = new Plan();
        plan->hs.assign(hs, hs + ninst);
        plan->xs.assign(xs, xs + ninst);
        plan->ys.assign(ys, ys + ninst);
        plan->dt = dt;
        plan->nvec = nvec;
        plan->st = st;
        for (int k = 0; k < ninst; ++k) {
            if (dt == XD_F32 && nvec == 8 && (int)plan->big.size() < kMaxBig8 && spmm8_usable(hs[k], xs[k], ys[k]))
                plan->big.push_back(k);
            else
                plan->rest.push_back(k);
        }
        xd_status s = autotune(plan);
        if (s == XD_OK) s = capture(plan);
        if (s != XD_OK) {
            free_plan(plan);
            return s;
        }
        g_plans.push_back(plan);
    }
    XD_CUDA(cudaGraphLaunch(plan->exec, st));
    return XD_OK;
}

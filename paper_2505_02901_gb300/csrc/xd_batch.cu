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
// autotuner that times every candidate once (CUDA events) the first time a
// batch is seen; the chosen launch is captured in a CUDA graph and replayed
// while the batch (handles, vectors, dtype, nvec, stream) is unchanged.
// Instances large enough for the prefix-block layout (N >= 24) with eight
// FP32 right-hand sides leave the persistent launch: each gets the
// eight-vector prefix-block product (xd_u1_spmm8.cu), in the same graph.

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "xd_internal.cuh"

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

template <typename T, int NV>
__global__ void k_batch(const Inst *__restrict__ inst, int ninst, int64_t ntiles, int tile_rows) {
    __shared__ uint64_t sm_mask[kMaxBatchBonds];
    __shared__ T sm_half[kMaxBatchBonds];
    __shared__ int sh_k;
    __shared__ uint64_t sh_range[2];
    int cur = -1;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = ninst - 1;  // last instance with tile0 <= t
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (inst[mid].tile0 <= t) lo = mid; else hi = mid - 1;
            }
            sh_k = lo;
        }
        __syncthreads();
        const int k = sh_k;
        const Inst &I = inst[k];
        const U1View &u = I.u;
        if (k != cur) {
            const uint64_t *masks = (const uint64_t *)(I.bond + I.nb);
            for (int b = threadIdx.x; b < I.nb; b += blockDim.x) {
                sm_mask[b] = masks[b];
                sm_half[b] = (T)(0.5 * I.bond[b]);
            }
            cur = k;
        }
        const int64_t row0 = (t - I.tile0) * tile_rows;
        const int64_t row1 = min(row0 + (int64_t)tile_rows, u.dim);
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
        __syncthreads();
    }
}

struct Plan {
    std::vector<const xd_ham_s *> hs;
    std::vector<const void *> xs;
    std::vector<void *> ys;
    std::vector<int> rest, big;  // instances of the persistent launch / of their own launch
    xd_dtype dt;
    int nvec;
    cudaStream_t st;
    Inst *d_inst = nullptr;
    int64_t ntiles = 0;
    int threads = 256, tile_rows = 1024, grid = 1;
    cudaGraphExec_t exec = nullptr;
    bool tuned = false;
};

std::mutex g_mu;
std::vector<Plan *> g_plans;

template <typename T, int NV>
void launch(const Plan &p, cudaStream_t st) {
    k_batch<T, NV><<<p.grid, p.threads, 0, st>>>(p.d_inst, (int)p.rest.size(), p.ntiles, p.tile_rows);
}

void launch_rest(const Plan &p, cudaStream_t st) {
    if (p.rest.empty()) return;
    if (p.dt == XD_F64) {
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
}

xd_status launch_any(const Plan &p, cudaStream_t st) {
    launch_rest(p, st);
    XD_CUDA(cudaGetLastError());
    for (int k : p.big) XD_TRY(spmm8_apply(p.hs[k], p.xs[k], p.ys[k], st));
    return XD_OK;
}

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
    if (h.empty()) return XD_OK;
    if (!p->d_inst) XD_CUDA(dev_malloc((void **)&p->d_inst, sizeof(Inst) * h.size()));
    XD_CUDA(cudaMemcpy(p->d_inst, h.data(), sizeof(Inst) * h.size(), cudaMemcpyHostToDevice));
    return XD_OK;
}

// Time each (threads, rows per tile) candidate once and keep the fastest.
xd_status autotune(Plan *p) {
    for (int k : p->big) XD_TRY(spmm8_apply(p->hs[k], p->xs[k], p->ys[k], p->st));  // attributes, warm
    if (p->rest.empty()) {
        p->tuned = true;
        return XD_OK;
    }
    const int cand_threads[] = {128, 256, 512};
    const int cand_rows_per_thread[] = {1, 4, 16};
    struct Events {  // destroyed on every return path
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    XD_CUDA(cudaEventCreate(&ev.a));
    XD_CUDA(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    float best = 1e30f;
    int bt = 256, br = 1024;
    for (int th : cand_threads)
        for (int rpt : cand_rows_per_thread) {
            p->threads = th;
            p->tile_rows = th * rpt;
            XD_TRY(build_table(p));
            p->grid = (int)std::max<int64_t>(1, std::min<int64_t>(p->ntiles, (int64_t)g_num_sms * (2048 / th)));
            launch_rest(*p, p->st);  // warm
            XD_CUDA(cudaEventRecord(e0, p->st));
            launch_rest(*p, p->st);
            XD_CUDA(cudaEventRecord(e1, p->st));
            XD_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            XD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bt = th;
                br = th * rpt;
            }
        }
    p->threads = bt;
    p->tile_rows = br;
    XD_TRY(build_table(p));
    p->grid = (int)std::max<int64_t>(1, std::min<int64_t>(p->ntiles, (int64_t)g_num_sms * (2048 / bt)));
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
            if (p->exec) cudaGraphExecDestroy(p->exec);
            cudaFree(p->d_inst);
            delete p;
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
            if (dt == XD_F32 && nvec == 8 && spmm8_usable(hs[k], xs[k], ys[k])) plan->big.push_back(k);
            else plan->rest.push_back(k);
        }
        xd_status s = autotune(plan);
        if (s == XD_OK) s = capture(plan);
        if (s != XD_OK) {
            if (plan->exec) cudaGraphExecDestroy(plan->exec);
            cudaFree(plan->d_inst);
            delete plan;
            return s;
        }
        g_plans.push_back(plan);
    }
    XD_CUDA(cudaGraphLaunch(plan->exec, st));
    return XD_OK;
}

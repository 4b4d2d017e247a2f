// xd_api.cu -- host side of the C ABI: validation, index tables, handles.
//
// Block construction follows Sec. 3.1 (U(1) blocks) and Sec. 3.9-3.10
// (groups, 1-D representations, symmetry-adapted blocks); the index layout
// is the two-table (Lin) scheme of Sec. 5.2 generalised to an arbitrary
// prefix/postfix split.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <set>
#include <string>
#include <unordered_map>

#include "xd_groups.h"
#include "xd_layout.h"
#include "xd_internal.cuh"

namespace xd {

static thread_local char g_err[512] = "no error";
int g_num_sms = 0;

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

// Injected allocation failure: -1 off; n >= 0: n more allocations succeed,
// the next one fails with cudaErrorMemoryAllocation (without allocating) and
// the injection switches itself off.
static std::atomic<int64_t> g_fail_after{-1};

cudaError_t dev_malloc(void **p, size_t bytes) {
    int64_t n = g_fail_after.load();
    while (n >= 0 && !g_fail_after.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

xd_status cuda_status(cudaError_t e, const char *what) {
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? XD_ENOMEM : XD_ECUDA;
}

int grid_for(int64_t work, int threads, int per_sm) {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    int64_t need = (work + threads - 1) / threads;
    int64_t cap = (int64_t)g_num_sms * per_sm;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

static int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;  // exact at each step
    return r;
}

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

template <typename T>
static xd_status dcopy(T **dst, const T *src, size_t n) {
    XD_CUDA(dev_malloc((void **)dst, std::max<size_t>(1, n) * sizeof(T)));
    if (n) XD_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return XD_OK;
}

cudaError_t dev_malloc_vec(xd_ham_s *h, void **p, size_t bytes) {
    cudaError_t e = dev_malloc(p, bytes);
    if (e == cudaErrorMemoryAllocation && h->d_x64_x) {
        cudaGetLastError();
        x64_release(h);
        e = dev_malloc(p, bytes);
    }
    return e;
}

xd_status ensure_partials(xd_ham_s *h, size_t bytes) {
    if (h->part_bytes >= bytes) return XD_OK;
    if (h->d_part) cudaFree(h->d_part);
    h->d_part = nullptr;
    h->part_bytes = 0;
    XD_CUDA(dev_malloc((void **)&h->d_part, bytes));
    h->part_bytes = bytes;
    return XD_OK;
}

static xd_status build_u1(xd_basis_s *b) {
    U1Layout lay;
    if (!u1_layout(b->N, b->nup, &lay)) {
        set_error("internal: U(1) layout size %lld != C(%d,%d)", (long long)lay.dim, b->N, b->nup);
        return XD_ERANGE;
    }
    b->L = lay.L;
    b->P = lay.P;
    b->dim_u1 = lay.dim;
    b->h_hi_off = std::move(lay.hi_off);
    b->h_lo_rank = std::move(lay.lo_rank);
    b->h_lo_list = std::move(lay.lo_list);
    b->h_lo_off = std::move(lay.lo_off);
    XD_TRY(dcopy(&b->d_hi_off, b->h_hi_off.data(), b->h_hi_off.size()));
    XD_TRY(dcopy(&b->d_lo_rank, b->h_lo_rank.data(), b->h_lo_rank.size()));
    XD_TRY(dcopy(&b->d_lo_list, b->h_lo_list.data(), b->h_lo_list.size()));
    XD_TRY(dcopy(&b->d_lo_off, b->h_lo_off.data(), b->h_lo_off.size()));
    return XD_OK;
}

static int64_t u1_index_host(const xd_basis_s *b, uint64_t s) {
    return u1_index(b->N, b->nup, b->L, b->h_hi_off, b->h_lo_rank, s);
}

static uint64_t u1_state_host(const xd_basis_s *b, int64_t idx) {
    return u1_state(b->nup, b->L, b->h_hi_off, b->h_lo_list, b->h_lo_off, idx);
}

// Group axioms and homomorphism (Sec. 3.9.1, Sec. 3.9.2), invariance of the
// bond graph.  Composition (f after g)(i) = f(g(i)).
static xd_status check_group(const xd_basis_s *b) {
    const int N = b->N, G = b->G;
    auto P = [&](int g) { return b->perms.data() + (size_t)g * N; };
    // permutation -> group index (the closure test is G^2 lookups)
    std::unordered_map<std::string, int> index;
    auto key = [&](const int32_t *p) { return std::string((const char *)p, sizeof(int32_t) * N); };
    for (int g = G - 1; g >= 0; --g) index[key(P(g))] = g;
    if ((int)index.size() != G) {
        set_error("symmetry: a permutation is listed more than once");
        return XD_ESYM;
    }
    auto find = [&](const int32_t *p) {
        auto it = index.find(key(p));
        return it == index.end() ? -1 : it->second;
    };
    std::vector<int32_t> t(N);
    bool has_id = false;
    for (int g = 0; g < G; ++g) {
        std::vector<char> seen(N, 0);
        bool id = true;
        for (int i = 0; i < N; ++i) {
            int v = P(g)[i];
            if (v < 0 || v >= N || seen[v]) {
                set_error("symmetry: row %d is not a permutation of 0..%d", g, N - 1);
                return XD_ESYM;
            }
            seen[v] = 1;
            id &= (v == i);
        }
        has_id |= id;
        if (fabs(hypot(b->chi_re[g], b->chi_im[g]) - 1.0) > 1e-9) {
            set_error("symmetry: |chi(g)| != 1 for g = %d", g);
            return XD_ESYM;
        }
    }
    if (!has_id) {
        set_error("symmetry: the identity permutation is missing");
        return XD_ESYM;
    }
    for (int f = 0; f < G; ++f)
        for (int g = 0; g < G; ++g) {
            for (int i = 0; i < N; ++i) t[i] = P(f)[P(g)[i]];
            int h = find(t.data());
            if (h < 0) {
                set_error("symmetry: not closed under composition (%d, %d)", f, g);
                return XD_ESYM;
            }
            double pr = b->chi_re[f] * b->chi_re[g] - b->chi_im[f] * b->chi_im[g];
            double pi = b->chi_re[f] * b->chi_im[g] + b->chi_im[f] * b->chi_re[g];
            if (fabs(pr - b->chi_re[h]) > 1e-9 || fabs(pi - b->chi_im[h]) > 1e-9) {
                set_error("symmetry: characters are not a homomorphism (%d, %d)", f, g);
                return XD_ESYM;
            }
        }
    for (int g = 0; g < G; ++g) {
        for (int i = 0; i < N; ++i) t[P(g)[i]] = i;
        if (find(t.data()) < 0) {
            set_error("symmetry: inverse of %d missing", g);
            return XD_ESYM;
        }
    }
    // the interaction graph must be invariant (as a multiset of pairs)
    std::multiset<std::pair<int, int>> E;
    for (auto &bd : b->bonds) E.insert({std::min(bd.i, bd.j), std::max(bd.i, bd.j)});
    for (int g = 0; g < G; ++g) {
        std::multiset<std::pair<int, int>> F;
        for (auto &bd : b->bonds) {
            int a = P(g)[bd.i], c = P(g)[bd.j];
            F.insert({std::min(a, c), std::max(a, c)});
        }
        if (F != E) {
            set_error("symmetry: permutation %d does not map the bond graph onto itself", g);
            return XD_ESYM;
        }
    }
    return XD_OK;
}

static void free_basis(xd_basis_s *b) {
    block_layout_free(b);
    spmm_layout_free(b);
    pass_layout_free(b);
    cudaFree(b->d_hi_off);
    cudaFree(b->d_lo_rank);
    cudaFree(b->d_lo_list);
    cudaFree(b->d_lo_off);
    cudaFree(b->d_reps);
    cudaFree(b->d_stab);
    cudaFree(b->d_rs);
    cudaFree(b->d_act);
    cudaFree(b->d_minrot);
    cudaFree(b->d_amask);
    cudaFree(b->d_rowtab);
    cudaFree(b->d_cut);
    cudaFree(b->d_krow);
    cudaFree(b->d_tg);
    cudaFree(b->d_tpp);
    cudaFree(b->d_pm);
    cudaFree(b->d_cg);
    cudaFree(b->d_chi);
    delete b;
}

}  // namespace xd

xd::U1View xd_basis_s::u1view() const {
    xd::U1View v;
    v.N = N;
    v.nup = nup;
    v.L = L;
    v.P = P;
    v.lomask = (1ull << L) - 1;
    v.dim = dim_u1;
    v.hi_off = d_hi_off;
    v.lo_rank = d_lo_rank;
    v.lo_list = d_lo_list;
    v.lo_off = d_lo_off;
    return v;
}

xd::SymView xd_basis_s::symview() const {
    xd::SymView v;
    v.N = N;
    v.G = G;
    v.dim = dim;
    v.reps = d_reps;
    v.stab = d_stab;
    v.rs = d_rs;
    v.act = d_act;
    v.nchunk = nchunk;
    v.u1 = u1view();
    v.tx = tx;
    v.ty = ty;
    v.minrot = d_minrot;
    v.amask = d_amask;
    v.rowtab = d_rowtab;
    v.cut = d_cut;
    v.krow = d_krow;
    v.trep1 = trep1;
    v.tg = d_tg;
    v.tnp = tnp;
    v.tpp = d_tpp;
    v.pm = d_pm;
    v.cn = cn;
    v.cdih = cdih;
    v.cg = d_cg;
    return v;
}

using namespace xd;

extern "C" {

const char *xd_last_error(void) { return xd::g_err; }

xd_status xd_debug_fail_alloc(int64_t n) {
    xd::g_fail_after.store(n < 0 ? -1 : n);
    return XD_OK;
}
const char *xd_version(void) { return "xdiag-gb300 0.1 (sm_103a)"; }

xd_status xd_basis_create(int N, int nup, const int32_t *bonds, int nb, const xd_symmetry *sym,
                          xd_basis *out) {
    if (!out) {
        set_error("xd_basis_create: out is NULL");
        return XD_EINVAL;
    }
    *out = nullptr;
    if (N < 2 || N > kMaxN) {
        set_error("xd_basis_create: N = %d outside [2, %d]", N, kMaxN);
        return N > kMaxN ? XD_ERANGE : XD_EINVAL;
    }
    if (nup < 0 || nup > N) {
        set_error("xd_basis_create: nup = %d outside [0, N]", nup);
        return XD_EINVAL;
    }
    if (!bonds || nb < 1 || nb > kMaxBonds) {
        set_error("xd_basis_create: need 1 <= nb <= %d bonds (got %d)", kMaxBonds, nb);
        return bonds && nb > kMaxBonds ? XD_ERANGE : XD_EINVAL;
    }
    for (int k = 0; k < nb; ++k) {
        int i = bonds[2 * k], j = bonds[2 * k + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j) {
            set_error("xd_basis_create: bond %d = (%d, %d) invalid for N = %d", k, i, j, N);
            return XD_EINVAL;
        }
    }
    int64_t dimu1 = binom(N, nup);
    if (dimu1 >= (1ll << 40)) {
        set_error("xd_basis_create: dimension %lld too large", (long long)dimu1);
        return XD_ERANGE;
    }
    auto *b = new xd_basis_s();
    b->N = N;
    b->nup = nup;
    b->nb = nb;
    for (int k = 0; k < nb; ++k) b->bonds.push_back({bonds[2 * k], bonds[2 * k + 1]});
    if (sym) {
        if (sym->ngroup < 1 || sym->ngroup > kMaxGroup || !sym->perms || !sym->chi_re ||
            !sym->chi_im) {
            set_error("xd_basis_create: symmetry needs 1 <= ngroup <= %d and non-NULL arrays",
                      kMaxGroup);
            delete b;
            return XD_EINVAL;
        }
        b->sym = true;
        b->G = sym->ngroup;
        b->perms.assign(sym->perms, sym->perms + (size_t)sym->ngroup * N);
        b->chi_re.assign(sym->chi_re, sym->chi_re + sym->ngroup);
        b->chi_im.assign(sym->chi_im, sym->chi_im + sym->ngroup);
        for (int g = 0; g < b->G; ++g) b->cplx |= fabs(b->chi_im[g]) > 1e-12;
        xd_status s = check_group(b);
        if (s != XD_OK) {
            delete b;
            return s;
        }
    }
    xd_status s = build_u1(b);
    if (s == XD_OK && b->sym) s = sym_build(b);
    if (s == XD_OK && block_layout_wanted(b)) s = block_layout_build(b);
    if (s == XD_OK && spmm_layout_wanted(b)) s = spmm_layout_build(b);
    if (s != XD_OK) {
        free_basis(b);
        return s;
    }
    if (!b->sym) b->dim = b->dim_u1;
    *out = b;
    return XD_OK;
}

xd_status xd_basis_dim(xd_basis b, int64_t *dim) {
    if (!b || !dim) {
        set_error("xd_basis_dim: NULL argument");
        return XD_EINVAL;
    }
    *dim = b->dim;
    return XD_OK;
}

xd_status xd_basis_is_complex(xd_basis b, int *c) {
    if (!b || !c) {
        set_error("xd_basis_is_complex: NULL argument");
        return XD_EINVAL;
    }
    *c = b->cplx ? 1 : 0;
    return XD_OK;
}

xd_status xd_basis_state(xd_basis b, int64_t idx, uint64_t *s) {
    if (!b || !s) {
        set_error("xd_basis_state: NULL argument");
        return XD_EINVAL;
    }
    if (idx < 0 || idx >= b->dim) {
        set_error("xd_basis_state: index %lld outside [0, %lld)", (long long)idx,
                  (long long)b->dim);
        return XD_ERANGE;
    }
    if (!b->sym) {
        *s = u1_state_host(b, idx);
        return XD_OK;
    }
    XD_CUDA(cudaMemcpy(s, b->d_reps + idx, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return XD_OK;
}

xd_status xd_basis_index(xd_basis b, uint64_t s, int64_t *idx) {
    if (!b || !idx) {
        set_error("xd_basis_index: NULL argument");
        return XD_EINVAL;
    }
    int64_t k = u1_index_host(b, s);
    if (!b->sym || k < 0) {
        *idx = k;
        return XD_OK;
    }
    ulonglong2 wc;
    XD_CUDA(cudaMemcpy(&wc, b->d_rs + (k >> 6), sizeof wc, cudaMemcpyDeviceToHost));
    const uint64_t w = wc.x;
    const int64_t c = (int64_t)wc.y;
    if (!((w >> (k & 63)) & 1)) {
        *idx = -1;
        return XD_OK;
    }
    *idx = c + popc64(w & ((1ull << (k & 63)) - 1));
    return XD_OK;
}

xd_status xd_basis_states(xd_basis b, int64_t first, int64_t count, uint64_t *out, xd_stream stream) {
    if (!b || (!out && count > 0)) {
        set_error("xd_basis_states: NULL argument");
        return XD_EINVAL;
    }
    if (first < 0 || count < 0 || first > b->dim || count > b->dim - first) {
        set_error("xd_basis_states: rows [%lld, %lld + %lld) outside 0..%lld", (long long)first, (long long)first,
                  (long long)count, (long long)b->dim);
        return XD_ERANGE;
    }
    if (count == 0) return XD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->sym) {
        XD_CUDA(cudaMemcpyAsync(out, b->d_reps + first, (size_t)count * sizeof(uint64_t), cudaMemcpyDefault, st));
        return XD_OK;
    }
    return u1_states(b, first, count, out, st);
}

void xd_basis_destroy(xd_basis b) {
    if (b) free_basis(b);
}

static xd_status set_J(xd_ham_s *h, const double *J) {
    const xd_basis_s *b = h->b;
    for (int k = 0; k < b->nb; ++k)
        if (!isfinite(J[k])) {
            set_error("coupling J[%d] is not finite", k);
            return XD_EINVAL;
        }
    if (b->sym) {
        // couplings must be invariant: J of a bond equals J of its image
        int g = 0, k = 0;
        if (!couplings_invariant(b->N, b->G, b->perms.data(), (const int32_t *)b->bonds.data(), b->nb, J, &g, &k)) {
            set_error("couplings are not invariant under permutation %d (bond %d)", g, k);
            return XD_ESYM;
        }
    }
    h->J.assign(J, J + b->nb);
    XD_CUDA(cudaMemcpy(h->d_J, J, sizeof(double) * b->nb, cudaMemcpyHostToDevice));
    std::vector<double> buf(2 * b->nb + 1);
    double q = 0.0;
    for (int k = 0; k < b->nb; ++k) {
        buf[k] = J[k];
        uint64_t m = (1ull << b->bonds[k].i) | (1ull << b->bonds[k].j);
        memcpy(&buf[b->nb + k], &m, sizeof m);
        q += J[k];
    }
    buf[2 * b->nb] = 0.25 * q;
    XD_CUDA(cudaMemcpy(h->d_bond, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice));
    if (b->sym && !h->d_symtab) XD_TRY(sym_ham_tables(h));
    if (b->sym) XD_TRY(sym_bond_groups(h));
    if (b->blk.ok) XD_TRY(block_ham_tables(h));
    if (b->spmm.ok) XD_TRY(spmm_ham_tables(h));
    if (b->spmm.ok) XD_TRY(passes_tables(h));
    lanczos_forget(h, false);
    batch_forget(h);  // captured batched launches hold per-coupling scalars
    return XD_OK;
}

xd_status xd_ham_create(xd_basis b, const double *J, xd_ham *out) {
    if (!b || !J || !out) {
        set_error("xd_ham_create: NULL argument");
        return XD_EINVAL;
    }
    *out = nullptr;
    auto *h = new xd_ham_s();
    h->b = b;
    cudaError_t e = dev_malloc((void **)&h->d_J, sizeof(double) * b->nb);
    if (e == cudaSuccess) e = dev_malloc((void **)&h->d_bond, sizeof(double) * (2 * b->nb + 1));
    if (e == cudaSuccess) e = dev_malloc((void **)&h->d_scal, sizeof(double) * 64);
    if (e != cudaSuccess) {
        cudaFree(h->d_J);
        cudaFree(h->d_bond);
        delete h;
        return cuda_status(e, "cudaMalloc(ham)");
    }
    xd_status s = set_J(h, J);
    if (s != XD_OK) {
        xd_ham_destroy(h);
        return s;
    }
    *out = h;
    return XD_OK;
}

xd_status xd_ham_set_couplings(xd_ham h, const double *J) {
    if (!h || !J) {
        set_error("xd_ham_set_couplings: NULL argument");
        return XD_EINVAL;
    }
    return set_J(h, J);
}

void xd_ham_destroy(xd_ham h) {
    if (!h) return;
    batch_forget(h);
    lanczos_forget(h, true);
    cudaFree(h->d_J);
    cudaFree(h->d_bond);
    cudaFree(h->d_lzpart);
    cudaFree(h->d_symtab);
    cudaFree(h->d_symgrp);
    cudaFree(h->d_dpost);
    cudaFree(h->d_sp_dpost);
    cudaFree(h->d_sp_jhalf);
    cudaFree(h->d_x64_tab);
    cudaFree(h->d_x64_x);
    cudaFree(h->d_x64_state);
    cudaFree(h->d_part);
    cudaFree(h->d_scal);
    delete h;
}

static xd_status check_vec_args(xd_ham h, const void *x, const void *y, xd_dtype dt, int nvec,
                                const char *who, bool alias_ok = false) {
    if (!h || !x || !y) {
        set_error("%s: NULL argument", who);
        return XD_EINVAL;
    }
    if (x == y && !alias_ok) {
        set_error("%s: x and y must be distinct buffers", who);
        return XD_EINVAL;
    }
    if (dt != XD_F64 && dt != XD_F32 && dt != XD_C128) {
        set_error("%s: unknown dtype %d", who, (int)dt);
        return XD_EINVAL;
    }
    if (nvec != 1 && nvec != 2 && nvec != 4 && nvec != 8) {
        set_error("%s: nvec = %d not in {1, 2, 4, 8}", who, nvec);
        return XD_EINVAL;
    }
    const xd_basis_s *b = h->b;
    if (b->cplx && dt != XD_C128) {
        set_error("%s: complex block needs XD_C128 vectors", who);
        return XD_EINVAL;
    }
    if (!b->sym && dt == XD_C128) {
        set_error("%s: XD_C128 is for complex symmetric blocks; use XD_F64/XD_F32", who);
        return XD_EINVAL;
    }
    if (b->sym && !b->cplx && dt == XD_C128) {
        set_error("%s: real symmetric block takes XD_F64 or XD_F32", who);
        return XD_EINVAL;
    }
    if (b->sym && nvec != 1) {
        set_error("%s: symmetric blocks take nvec = 1", who);
        return XD_EINVAL;
    }
    if (b->sym && dt == XD_F32) {
        set_error("%s: symmetric blocks take XD_F64 (real) or XD_C128", who);
        return XD_EINVAL;
    }
    return XD_OK;
}

xd_status xd_apply(xd_ham h, const void *x, void *y, xd_dtype dt, int nvec, xd_stream stream) {
    XD_TRY(check_vec_args(h, x, y, dt, nvec, "xd_apply"));
    if (h->b->dim == 0) return XD_OK;
    if (h->b->sym) return sym_apply(h, x, y, dt, (cudaStream_t)stream);
    return u1_apply(h, x, y, dt, nvec, (cudaStream_t)stream);
}

xd_status xd_apply_bilinear(xd_ham h, const void *g, const void *x, xd_dtype dt, double *dJ,
                            xd_stream stream) {
    if (!dJ) {
        set_error("xd_apply_bilinear: dJ is NULL");
        return XD_EINVAL;
    }
    if (!h || !g || !x) {
        set_error("xd_apply_bilinear: NULL argument");
        return XD_EINVAL;
    }
    XD_TRY(check_vec_args(h, g, x, dt, 1, "xd_apply_bilinear", true));
    if (h->b->sym) return sym_bilinear(h, g, x, dt, dJ, (cudaStream_t)stream);
    return u1_bilinear(h, g, x, dt, dJ, (cudaStream_t)stream);
}

xd_status xd_apply_bilinear_nvec(xd_ham h, const void *g, const void *x, xd_dtype dt, int nvec, double *dJ,
                                 xd_stream stream) {
    if (!dJ || !h || !g || !x) {
        set_error("xd_apply_bilinear_nvec: NULL argument");
        return XD_EINVAL;
    }
    XD_TRY(check_vec_args(h, g, x, dt, nvec, "xd_apply_bilinear_nvec", true));
    if (nvec == 1) return xd_apply_bilinear(h, g, x, dt, dJ, stream);
    return u1_bilinear_nvec(h, g, x, dt, nvec, dJ, (cudaStream_t)stream);
}

xd_status xd_random_vector(int64_t dim, uint64_t seed, void *out, xd_dtype dt,
                           xd_stream stream) {
    if (!out || dim < 0) {
        set_error("xd_random_vector: bad argument");
        return XD_EINVAL;
    }
    if (dt != XD_F64 && dt != XD_F32 && dt != XD_C128) {
        set_error("xd_random_vector: unknown dtype");
        return XD_EINVAL;
    }
    return vec_random(dim, seed, out, dt, (cudaStream_t)stream);
}

}  // extern "C"

// xd_internal.cuh -- shared declarations of the CUDA library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "xdiag_gpu.h"

namespace xd {

// ------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
xd_status cuda_status(cudaError_t e, const char *what);

#define XD_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::xd::cuda_status(e_, #call);          \
    } while (0)

#define XD_TRY(call)                                                         \
    do {                                                                     \
        xd_status s_ = (call);                                               \
        if (s_ != XD_OK) return s_;                                          \
    } while (0)

constexpr int kMaxBonds = 4096;

// cudaMalloc, unless an allocation failure was injected (xd_debug_fail_alloc):
// every device allocation of the library goes through here.
cudaError_t dev_malloc(void **p, size_t bytes);
constexpr int kMaxGroup = 2048;
constexpr int kMaxN = 40;

// ----------------------------------------------------- U(1) index layout
// A state word s splits into a prefix h = s >> L (P = N - L bits) and a
// postfix l = s & (2^L - 1).  Rows with the same prefix form one contiguous
// block (ascending l inside, blocks ascending in h), so
//     index(s) = hi_off[h] + lo_rank[l]
// where hi_off[h] is the first row of block h and lo_rank[l] the rank of l
// among the L-bit words of its popcount (the two Lin tables of Sec. 5.2).
// lo_list lists the L-bit words sorted by (popcount, value); class m starts
// at lo_off[m].
struct U1View {
    int N, nup, L, P;
    uint64_t lomask;
    int64_t dim;
    const int64_t *hi_off;    // [2^P + 1], hi_off[2^P] = dim
    const uint32_t *lo_rank;  // [2^L]
    const uint32_t *lo_list;  // [2^L]
    const uint32_t *lo_off;   // [L + 2]
};

// ------------------------------------------------- symmetric block view
// Representatives ascending; membership of a U(1) word is a rank/select
// bitmap over U(1) ranks: bit k of bits is set when U(1) state k is a
// representative in the block, cum[w] counts the set bits before word w.
struct SymView {
    int N, G;
    int64_t dim;
    const uint64_t *reps;   // [dim]
    const uint16_t *stab;   // [dim] |Stab(r)|
    const ulonglong2 *rs;   // [ceil(dimU1 / 64)]: (member bits, members before the word)
    const uint64_t *act;    // [G][nchunk][256] byte tables of the action
    int nchunk;
    U1View u1;
    // translation group of an Lx x Ly torus (site x + Lx*y) inside the group,
    // when detected: tx = Lx (0 otherwise), ty = Ly; minrot/amask: smallest
    // rotation of an Lx-bit row and the rotations reaching it.  The group is
    // the union of the cosets T p_k (k < max(1, tnp)); tpp[k] = group index of
    // p_k, p_0 the identity; tg[k Lx Ly + a + Lx b] = group index of the
    // element s -> T_{a,b}(p_k s).  tnp = 0: translations only.
    int tx, ty, tnp;
    const uint8_t *minrot, *amask;
    // rowtab[r] = minrot[r] | amask[r] << 8; trep1 = bit 0 of every row;
    // cut: the narrowing search's row table (tx <= 7, else null; xd_orbit.h);
    // krow[k nb + b] = the rows of the two sites of p_k applied to bond b
    // (low byte, high byte), k < max(1, tnp), p_0 the identity
    const uint16_t *rowtab, *cut, *krow;
    uint64_t trep1;
    const int16_t *tg, *tpp;
    // pm[(k - 1) nb + b] = p_k applied to the mask of bond b (k >= 1): the
    // action is linear over XOR, so p_k(s ^ m) = p_k(s) ^ p_k(m)
    const uint64_t *pm;
    // rotations of a ring (i -> i + n mod N), with or without the reflections
    // (i -> n - i mod N), when detected: cn = N (0 otherwise), cdih = 1 with
    // reflections; cg[n] = group index of rotation n, cg[N + n] of reflection n
    int cn, cdih;
    const int16_t *cg;
};

struct Bond {
    int i, j;
};
// a bond list is read as [nb][2] int32 site pairs (xd_groups.h)
static_assert(sizeof(Bond) == 2 * sizeof(int32_t), "Bond is two int32 sites");

// Block-structured layout of a large U(1) block (xd_u1_block.cu).
struct BlockLayoutHost {
    bool ok = false;
    int npre = 0, ncross = 0, npost = 0, npost_pad = 0;
    int64_t nblk = 0;             // non-empty prefix blocks
    int maxblk = 0;               // largest block, C(L, L/2)
    std::vector<int> post;        // postfix bond ids
    uint32_t *d_order = nullptr;  // non-empty prefixes, ascending
    uint16_t *d_ptab = nullptr;   // postfix flip targets, bond-major
    uint16_t *d_xtab = nullptr;   // cross flip targets per postfix site
    int32_t *d_postid = nullptr;
    int32_t *d_pre = nullptr, *d_cross = nullptr, *d_csite = nullptr;
    int ncsite = 0;
};

// Batched FP32 layout of a large U(1) block (xd_u1_spmm.cu).
struct SpmmLayoutHost {
    bool ok = false;
    int L = 0, P = 0, npost = 0, npost_pad = 0, npre = 0, ncross = 0, ncsite = 0, maxblk = 0, maxpa = 0;
    int64_t nitems = 0;
    std::vector<uint32_t> h_lo_off, h_lo_list;
    std::vector<int> post, cross_ids;
    int64_t *d_hi_off = nullptr, *d_pcsr_off = nullptr;
    uint32_t *d_lo_off = nullptr, *d_lo_list = nullptr, *d_lo_rank = nullptr, *d_items = nullptr;
    uint16_t *d_ptab = nullptr, *d_xtab = nullptr, *d_postid = nullptr;
    int32_t *d_pre = nullptr, *d_cross = nullptr, *d_csite = nullptr;
    uint64_t *d_pcsr = nullptr;
    std::vector<int32_t> h_pre, h_csite;  // prefix bond triples, cross site triples
};

// Passes of the prefix bonds and the work items of the product in passes
// (xd_u1_passes.cu), built on first use.
struct PassLayoutHost {
    bool ok = false, unusable = false;   // unusable: the prefix bonds need more than four windows
    int npass = 0;
    int ws[4] = {}, nwb[4] = {};         // window bits and bonds of each pass
    uint16_t *d_wlist[4] = {}, *d_wrank[4] = {};  // window words by (popcount, value); their ranks
    uint32_t *d_woff[4] = {}, *d_wdep[4] = {};    // first word per popcount; deposited prefix bits
    uint32_t *d_wbond[4] = {};           // window mask | bond << 16
    uint64_t *d_pitems[4] = {};          // other prefix bits | window popcount << 32 | rank chunk << 40
    int64_t nitems_p[4] = {};
    std::vector<int> cross_low;          // prefix sites of the cross bonds (lowest in the items' key)
    uint32_t *d_items[2] = {};           // k_main's items of 4 and of 8 same-class prefixes
    int64_t nitems[2] = {};
};

}  // namespace xd

struct xd_basis_s {
    int N = 0, nup = 0, nb = 0;
    std::vector<xd::Bond> bonds;
    // U(1) layout (always present; a symmetric block uses it for ranks)
    int L = 0, P = 0;
    int64_t dim_u1 = 0;
    std::vector<int64_t> h_hi_off;
    std::vector<uint32_t> h_lo_rank, h_lo_list, h_lo_off;
    int64_t *d_hi_off = nullptr;
    uint32_t *d_lo_rank = nullptr, *d_lo_list = nullptr, *d_lo_off = nullptr;
    // symmetric block
    bool sym = false, cplx = false;
    int G = 0;
    std::vector<int32_t> perms;
    std::vector<double> chi_re, chi_im;
    int64_t dim = 0;
    uint64_t *d_reps = nullptr;
    uint16_t *d_stab = nullptr;
    ulonglong2 *d_rs = nullptr;      // rank/select words: (bits, count before)
    uint64_t *d_act = nullptr;
    int nchunk = 0;
    int tx = 0, ty = 0, tnp = 0;     // detected torus translations (and their cosets)
    uint8_t *d_minrot = nullptr, *d_amask = nullptr;
    uint16_t *d_rowtab = nullptr, *d_cut = nullptr, *d_krow = nullptr;
    uint64_t trep1 = 0;
    int16_t *d_tg = nullptr, *d_tpp = nullptr;
    uint64_t *d_pm = nullptr;        // point images of the bond masks
    int cn = 0, cdih = 0;            // detected ring rotations (+ reflections)
    int16_t *d_cg = nullptr;
    double *d_chi = nullptr;  // [G][2]
    xd::BlockLayoutHost blk;
    xd::SpmmLayoutHost spmm;
    xd::PassLayoutHost pass;

    xd::U1View u1view() const;
    xd::SymView symview() const;
};

struct xd_ham_s {
    xd_basis b = nullptr;
    std::vector<double> J;
    double *d_J = nullptr;          // [nb]
    double *d_bond = nullptr;       // [J (nb) | bond masks (nb, as uint64) | sum J / 4]
    double *d_part = nullptr;       // reduction partials
    size_t part_bytes = 0;
    double *d_scal = nullptr;       // small device scalars
    double *d_lzpart = nullptr;     // Lanczos reduction partials
    int lzpart_n = 0;
    double *d_symtab = nullptr;     // symmetric blocks: sqrt(a), 1/sqrt(a) [G+1 each] | bond orbit ids
    // symmetric blocks: bonds sorted by coupling, in chunks of 64 split into
    // groups of equal coupling (sym_bond_groups): [nb] masks | [ngrp] group
    // masks | [ngrp] J/2 | [nb] u16 bond ids | [nchunk + 1] u16 first groups
    uint64_t *d_symgrp = nullptr;
    int sym_ngrp = 0;
    double *d_dpost = nullptr;      // block layout: postfix diagonal per L-bit word
    float *d_sp_dpost = nullptr;    // batched layout: postfix diagonal per class position
    float *d_sp_jhalf = nullptr;    // batched layout: J/2 per bond
    float sp_jcross = 0.f;          // batched layout: sum over cross bonds of J/4
    // FP64 product on the batched layout without FP64 arithmetic per element
    // (xd_u1_passes.cu): fixed point when the couplings are small integer
    // multiples of one quantum, else double-float
    bool x64_fx_ok = false;         // the couplings have a quantum: fixed point allowed
    void *d_x64_tab = nullptr;      // one allocation holding the tables below
    void *d_x64_dfc = nullptr, *d_x64_dfd = nullptr, *d_x64_dfp = nullptr;  // double-float: J/2, J/4, postfix diagonal
    void *d_x64_fxc = nullptr, *d_x64_fxd = nullptr, *d_x64_fxp = nullptr;  // fixed point: 2 k_b, k_b, postfix D
    uint32_t *d_x64_post = nullptr; // postfix bond masks | bond << 16
    double x64_dcross_d = 0.0, x64_qs = 1.0;
    int x64_dcross_i = 0, x64_B = 0;
    void *d_x64_x = nullptr;        // workspace, 8 bytes per row (allocated on first use)
    int *d_x64_state = nullptr;     // [E, mode] and the statistics partials
    // first Lanczos pass (xd_lanczos.cu): its stream, device state and, for
    // small blocks, the captured steps with their three vectors (dropped when
    // the couplings change: the captured kernels hold values derived from them)
    cudaStream_t lz_stream = nullptr;
    void *lz_dstate = nullptr, *lz_hstate = nullptr;
    double *lz_ab = nullptr;
    int lz_ab_cap = 0;
    cudaGraphExec_t lz_exec = nullptr;
    void *lz_buf[3] = {nullptr, nullptr, nullptr};
    int lz_key_dt = -1, lz_key_iter = 0;
};

namespace xd {

// ------------------------------------------------------------ kernels
// U(1) product (xd_u1.cu)
xd_status u1_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt,
                   int nvec, cudaStream_t st);
xd_status u1_bilinear(const xd_ham_s *h, const void *g, const void *x,
                      xd_dtype dt, double *dJ, cudaStream_t st);
xd_status u1_states(const xd_basis_s *b, int64_t first, int64_t count, uint64_t *out, cudaStream_t st);
xd_status u1_bilinear_nvec(const xd_ham_s *h, const void *g, const void *x, xd_dtype dt, int nv, double *dJ,
                           cudaStream_t st);
// symmetric blocks (xd_sym.cu)
xd_status sym_build(xd_basis_s *b);
xd_status sym_ham_tables(xd_ham_s *h);
xd_status sym_bond_groups(xd_ham_s *h);  // on every new set of couplings
xd_status sym_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt,
                    cudaStream_t st);
xd_status sym_bilinear(const xd_ham_s *h, const void *g, const void *x,
                       xd_dtype dt, double *dJ, cudaStream_t st);
xd_status sym_correlations(const xd_basis_s *b, const void *psi, xd_dtype dt, const int32_t *pairs, int npairs,
                           int kind, double *out);
// vector kernels (xd_vec.cu)
xd_status vec_random(int64_t n, uint64_t seed, void *out, xd_dtype dt,
                     cudaStream_t st);
// block-structured U(1) product (xd_u1_block.cu)
bool block_layout_wanted(const xd_basis_s *b);
xd_status block_layout_build(xd_basis_s *b);
void block_layout_free(xd_basis_s *b);
xd_status block_ham_tables(xd_ham_s *h);
xd_status block_apply(const xd_ham_s *h, const void *x, void *y, xd_dtype dt, cudaStream_t st);
// batched FP32 U(1) product (xd_u1_spmm.cu)
bool spmm_layout_wanted(const xd_basis_s *b);
xd_status spmm_layout_build(xd_basis_s *b);
void spmm_layout_free(xd_basis_s *b);
xd_status spmm_ham_tables(xd_ham_s *h);
xd_status spmm_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st);
// FP64 product in passes over prefix blocks on the same layout, fixed point
// or double-float (xd_u1_passes.cu)
xd_status passes_tables(xd_ham_s *h);
bool passes_usable(const xd_ham_s *h);
xd_status passes_apply_f64(const xd_ham_s *h, const void *x, void *y, cudaStream_t st);
void pass_layout_free(xd_basis_s *b);
// free the FP64 product's workspace (the next FP64 product allocates it again)
void x64_release(xd_ham_s *h);
// device allocation for a driver's vectors: when it fails, the handle's FP64
// product workspace is released and the allocation tried once more
cudaError_t dev_malloc_vec(xd_ham_s *h, void **p, size_t bytes);
// eight right-hand sides on the same layout (xd_u1_spmm8.cu); x, y [dim][8] FP32
bool spmm8_usable(const xd_ham_s *h, const void *x, const void *y);
xd_status spmm8_apply(const xd_ham_s *h, const void *x, void *y, cudaStream_t st);
// forget cached batch plans that use this handle (xd_batch.cu)
void batch_forget(const xd_ham_s *h);
// drop the first Lanczos pass's captured steps (and with all = true its stream
// and buffers) (xd_lanczos.cu)
void lanczos_forget(xd_ham_s *h, bool all);
// workspace helper
xd_status ensure_partials(xd_ham_s *h, size_t bytes);

int grid_for(int64_t work, int threads, int per_sm);
extern int g_num_sms;

}  // namespace xd

/*
 * xdiag_gpu.h -- C ABI of the GB300 matrix-free spin-1/2 Heisenberg library.
 *
 * The operation is the product y = H x of XDiag's Lanczos iteration
 * (Sec. 3.5 "apply", Sec. 5.1 apply_terms), for
 *     H = sum_b J_b S_{i_b} . S_{j_b}                      (Eq. 1, App. A SdotS)
 * on a block of fixed magnetisation (Spinhalf(N, nup), Sec. 3.1) or on a
 * symmetry-adapted block of a 1-D representation of a site-permutation group
 * (Spinhalf(N, nup, irrep), Sec. 3.9-3.10).  Around it: the Lanczos
 * eigensolver (eigval0 / eigvals_lanczos / eig0, Sec. 3.6.1), per-bond
 * expectation values (inner, Sec. 3.7) used as dE0/dJ_b, and a batched
 * product over many independent blocks (the multi-vector apply of Sec. 5.1).
 *
 * Conventions
 *   - Bit i of a state word is site i; a set bit is an up spin.  The U(1)
 *     block lists every N-bit word with nup set bits in ascending order with
 *     0-based indices (Sec. 3.1).  A symmetric block lists the
 *     representatives (the smallest integer of each orbit, Sec. 3.10) whose
 *     projected state does not vanish, ascending.
 *   - A permutation g acts by (g s)_i = s_{g(i)}; the basis state of the
 *     representative r is (1/N_r) sum_g conj(chi(g)) g|r>,
 *     N_r = sqrt(|G| |Stab(r)|) (Sec. 3.10).
 *   - Vectors are device arrays in the caller's memory, row-major
 *     [dim][nvec]; complex vectors interleave (re, im) doubles.
 *
 * Ownership and errors
 *   - The caller owns every vector it passes (x, y, g, psi0).  The library
 *     owns its index tables and workspaces; *_destroy frees them.
 *   - Every call returns an xd_status; nothing throws across the ABI.  On an
 *     error the thread-local message of xd_last_error() says why.  Inputs
 *     are validated before anything is launched.
 *   - Calls that take a cudaStream_t are asynchronous on that stream (NULL
 *     is the legacy default stream); calls that return host scalars
 *     synchronise.
 *   - A handle may be used from one host thread at a time.
 */
#ifndef XDIAG_GPU_H
#define XDIAG_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *xd_stream; /* same type as cudaStream_t */

typedef enum {
    XD_OK = 0,
    XD_EINVAL = 1,   /* bad argument (N, nup, bonds, dtype, null pointer, ...) */
    XD_ERANGE = 2,   /* a size or index beyond what the library supports     */
    XD_ENOMEM = 3,   /* device or host allocation failed                       */
    XD_ECUDA = 4,    /* a CUDA runtime call or kernel failed                   */
    XD_ESYM = 5,     /* not a group, not a homomorphism, H not invariant       */
    XD_ENOTCONV = 6  /* Lanczos stopped without meeting its criterion          */
} xd_status;

typedef enum {
    XD_F64 = 0,  /* double vectors                                          */
    XD_F32 = 1,  /* float vectors (storage); products and sums in FP32,
                    Lanczos dots and alpha/beta in FP64-class arithmetic     */
    XD_C128 = 2  /* complex double vectors, interleaved (re, im)            */
} xd_dtype;

/* A finite group of site permutations with a 1-D representation
 * (Sec. 3.9.1-3.9.2).  perms is [ngroup][N] with perms[g][i] = g(i);
 * chi_re/chi_im are the characters chi(g).  Validated: every row is a
 * permutation, no row is listed twice, the identity is present, the set is
 * closed under composition and inverses, chi is a homomorphism with
 * |chi| = 1, and the bond graph (with its couplings) is mapped onto itself.
 * Any element order is accepted.  The orbit search is fastest when the
 * group holds all translations of an Lx x Ly torus (site x + Lx*y, Lx <= 8):
 * alone, or with point operations (the group is then searched coset by
 * coset); the rotations of a ring, with or without its reflections, have a
 * fast search too; other groups take a search over every element. */
typedef struct {
    int ngroup;
    const int32_t *perms;
    const double *chi_re;
    const double *chi_im;
} xd_symmetry;

typedef struct xd_basis_s *xd_basis;
typedef struct xd_ham_s *xd_ham;

/* ---------------------------------------------------------------- basis */

/* Create the block Spinhalf(N, nup[, irrep]) (Sec. 3.1, Sec. 3.10) for the
 * interaction graph `bonds` ([nb][2] site pairs, 0-based, i != j, host
 * memory).  sym == NULL gives the U(1) block.  The graph decides the index
 * layout; its couplings are set by xd_ham_create.
 * Limits: 2 <= N <= 40 for U(1) blocks, N <= 40 and ngroup <= 2048 for
 * symmetric ones, 1 <= nb <= 4096, dim < 2^40.  Errors: XD_EINVAL,
 * XD_ERANGE, XD_ESYM, XD_ENOMEM, XD_ECUDA. */
xd_status xd_basis_create(int N, int nup, const int32_t *bonds, int nb,
                          const xd_symmetry *sym, xd_basis *out);

/* Number of basis states (rows of H). */
xd_status xd_basis_dim(xd_basis b, int64_t *dim);

/* 1 when vectors of this block are complex (a symmetric block whose
 * characters are not all real), else 0. */
xd_status xd_basis_is_complex(xd_basis b, int *is_complex);

/* State word of index idx (Sec. 3.1 "index" inverse); XD_ERANGE if out of
 * range.  Host call, synchronous. */
xd_status xd_basis_state(xd_basis b, int64_t idx, uint64_t *s);

/* Index of state word s, or -1 when s is not a basis state (for a
 * symmetric block: s must be a representative).  Host call. */
xd_status xd_basis_index(xd_basis b, uint64_t s, int64_t *idx);

/* State words of the rows [first, first + count) of the block, in row
 * order (Sec. 3.1: the block's basis states; for a symmetric block its
 * representatives, Sec. 3.10), written to out [count] uint64 in device (or
 * host-pinned) memory, caller-owned.  XD_ERANGE when the range leaves the
 * block.  Asynchronous on `stream`. */
xd_status xd_basis_states(xd_basis b, int64_t first, int64_t count,
                          uint64_t *out, xd_stream stream);

void xd_basis_destroy(xd_basis b);

/* ---------------------------------------------------------- Hamiltonian */

/* H = sum_b J_b S_i.S_j on basis b (Eq. 1); J is [nb] host doubles.  For a
 * symmetric block the couplings must be invariant under the group. */
xd_status xd_ham_create(xd_basis b, const double *J, xd_ham *out);

/* Replace the couplings (same validation as create). */
xd_status xd_ham_set_couplings(xd_ham h, const double *J);

void xd_ham_destroy(xd_ham h);

/* y = H x (Sec. 3.5 apply; Sec. 5.1 apply_terms with the vector "fill").
 * x, y: device arrays [dim][nvec] of dtype, distinct, caller-owned.
 * nvec in {1, 2, 4, 8} (nvec > 1: XD_F32 or XD_F64 on U(1) blocks).
 * XD_C128 is required on complex blocks; real blocks take XD_F64/XD_F32.
 * Asynchronous on `stream`. */
xd_status xd_apply(xd_ham h, const void *x, void *y, xd_dtype dtype,
                   int nvec, xd_stream stream);

/* Per-bond bilinear forms dJ[b] = Re <g| S_{i_b}.S_{j_b} |x> for every bond
 * (the J_b-derivative of Re <g|H|x>; Sec. 3.7 inner).  g, x: device [dim]
 * vectors of dtype (nvec = 1); dJ: device [nb] doubles.  The sum over rows
 * is deterministic (fixed-order two-stage reduction).  Asynchronous. */
xd_status xd_apply_bilinear(xd_ham h, const void *g, const void *x,
                            xd_dtype dtype, double *dJ, xd_stream stream);

/* Per-bond bilinear forms summed over nvec columns: dJ[b] = sum_k Re <g_k|
 * S_{i_b}.S_{j_b} |x_k> for row-major [dim][nvec] device arrays g, x (the
 * J_b-derivative of Re sum_k <g_k|H|x_k>, the backward of a product on a
 * block of vectors; Sec. 3.7 inner, Sec. 5.1 multi-vector apply).  nvec in
 * {1, 2, 4, 8}; nvec > 1 on U(1) blocks with XD_F64 or XD_F32.  dJ: device
 * [nb] doubles.  Every column is reduced in a fixed order and the columns are
 * summed in a fixed order (deterministic).  Asynchronous. */
xd_status xd_apply_bilinear_nvec(xd_ham h, const void *g, const void *x,
                                 xd_dtype dtype, int nvec, double *dJ,
                                 xd_stream stream);

/* Same per-bond bilinear forms as xd_apply_bilinear, for callers that must
 * not have the library allocate device memory: a process whose allocator
 * owns all of the GPU's memory (a pool or a fixed budget set at start-up),
 * or a latency-sensitive loop where cudaMalloc/cudaFree may synchronise the
 * device.  This call allocates nothing: its partial sums live in one fixed
 * array of 608 x 256 doubles (1.19 MiB) inside the library, which every GPU
 * that loads the library keeps until the process exits.  The paper has no
 * counterpart; it is an interface convenience of this library.
 * U(1) blocks only; dtype XD_F64 or XD_F32; g, x device [dim] vectors;
 * dJ device [nb] doubles, caller-owned.  Blocks with more than 256 bonds are
 * rejected with XD_ERANGE (xd_apply_bilinear has no such limit).
 * The first call on each device looks up that array's device address (this
 * may load the library's device code on that device); make that first call
 * before any stream capture.  The address is cached per device index for
 * the life of the process: after a cudaDeviceReset the cached address is
 * stale, so do not use this call in a process that resets its devices.  All calls share the array and it keeps the
 * last call's contents, so calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Asynchronous
 * on `stream`. */
xd_status xd_apply_bilinear_noalloc(xd_ham h, const void *g, const void *x,
                                    xd_dtype dtype, double *dJ, xd_stream stream);

/* Two-point spin correlations of a state (the expectation values of Sec. 3.7
 * inner, with the SzSz / SdotS operators of App. A on arbitrary site pairs):
 * out[p] = <psi| O |psi> for pair p = (i_p, j_p), O = Sz_i Sz_j (kind 0) or
 * S_i.S_j (kind 1); i = j is allowed ((Sz_i)^2 = 1/4, S_i.S_i = 3/4 times
 * <psi|psi>).  psi is not normalised by the call.  U(1) blocks: psi a device
 * [dim] vector of XD_F64 or XD_F32.  Symmetry-adapted blocks (Sec. 3.10):
 * psi of XD_F64 (real block) or XD_C128 (complex block), the value is that
 * of the lifted state |psi> = sum_r psi_r |r_chi>; within a one-dimensional
 * irrep it is the same on every pair of an orbit of the group, and the call
 * forms it from the symmetric bond form of the pair's orbit on the block's
 * own representatives.  pairs: host [npairs][2] site indices in [0, N); out:
 * host [npairs] doubles.  Sums run in FP64 in a fixed order
 * (deterministic).  Synchronous; allocates its workspace per call. */
xd_status xd_correlations(xd_basis b, const void *psi, xd_dtype dtype,
                          const int32_t *pairs, int npairs, int kind,
                          double *out);

/* ---------------------------------------------------------------- Lanczos */

/* Lanczos tridiagonalisation from the seeded normal start vector
 * (Sec. 3.5 random_state, Sec. 3.6.1 eigvals_lanczos).  Runs at most
 * max_iter steps, stopping early when beta_k < 1e-13 max|alpha|; vectors
 * are stored in `storage` (XD_F64, XD_F32, or XD_C128 on complex blocks),
 * dot products and alpha/beta in FP64-class arithmetic.  Host outputs:
 * alpha[max_iter], beta[max_iter], *n_iter, evals[nev] (lowest Ritz
 * values), resid[nev] (|beta_k * last component of the Ritz vector|).
 * Synchronous.  Device workspace: three vectors of `storage`. */
xd_status xd_lanczos_eigenvalues(xd_ham h, int max_iter, uint64_t seed,
                                 xd_dtype storage, int nev, double *alpha,
                                 double *beta, int *n_iter, double *evals,
                                 double *resid);

/* As above, then a second Lanczos pass from the same start that rebuilds
 * the lowest Ritz vector (eig0, Sec. 3.6.1) into psi0 (device, caller-
 * owned, [dim] of `storage`, unit norm). */
xd_status xd_lanczos_ground_state(xd_ham h, int max_iter, uint64_t seed,
                                  xd_dtype storage, int nev, double *alpha,
                                  double *beta, int *n_iter, double *evals,
                                  double *resid, void *psi0);

/* Time evolution out = exp(-z H) psi0 with z = z_re + i z_im (Sec. 3.6.2:
 * z = i t is the real-time evolution e^{-iHt}, z = tau the imaginary-time
 * e^{-tau H}), by the memory-efficient two-pass Lanczos method the paper
 * uses: pass 1 builds the tridiagonal T_m from psi0/|psi0| until the error
 * estimate |psi0| beta_m |[exp(-z T_m) e_1]_m| is at most tol |psi0| (or
 * max_iter steps), pass 2 repeats the recurrence and sums the Krylov vectors
 * with the coefficients |psi0| exp(-z T_m) e_1.
 * psi0, out: distinct device [dim] complex vectors (interleaved re, im
 * doubles) on any block; 1 <= max_iter <= 1000.  Host outputs: *n_iter = m,
 * *err = the final error estimate (absolute).  Synchronous.  Device
 * workspace: three complex vectors. */
xd_status xd_evolve(xd_ham h, const void *psi0, double z_re, double z_im,
                    int max_iter, double tol, void *out, int *n_iter,
                    double *err);

/* Finite-temperature Lanczos / thermal pure quantum states (the
 * thermodynamics examples of Sec. 4, Sugiura-Shimizu TPQ and the FTLM of
 * Jaklic-Prelovsek): R seeded random start vectors (start r is the
 * standard-normal vector of xd_random_vector with seed + r), each run
 * through M plain Lanczos steps (a run whose beta drops below 1e-13
 * max|alpha| stops early).  U(1) blocks run eight starts at a time through
 * the eight-vector product (device workspace: three [dim][8] FP64 arrays);
 * symmetry-adapted blocks run one Lanczos pass per start on the block's own
 * product (complex vectors on complex blocks; workspace: three vectors).
 * Host outputs: alpha, beta [R][M] (zero past n_iter[r]), n_iter [R].
 * Synchronous. */
xd_status xd_ftlm(xd_ham h, int R, int M, uint64_t seed, double *alpha,
                  double *beta, int *n_iter);

/* Thermodynamics from the tridiagonals of xd_ftlm (host only): with T_r =
 * Q diag(eps) Q^T and weights |Q_0j|^2, at each temperature T[q] > 0
 *   Z = (dim / R) sum_{r,j} |Q_0j|^2 e^{-eps_j/T},  E = <eps>,  C = (<eps^2> - E^2) / T^2.
 * Outputs Z, E, C: host [nT]. */
xd_status xd_ftlm_thermo(int R, int M, const double *alpha, const double *beta,
                         const int *n_iter, double dim, int nT,
                         const double *temps, double *Z, double *E, double *C);

/* dE0/dJ_b = <psi0| S_{i_b}.S_{j_b} |psi0> (Hellmann-Feynman with the
 * expectation values of Sec. 3.7); psi0 is a device unit vector of dtype;
 * dEdJ is [nb] host doubles.  Synchronous. */
xd_status xd_energy_grad(xd_ham h, const void *psi0, xd_dtype dtype,
                         double *dEdJ);

/* Seeded standard-normal vector (the random_state of Sec. 3.5 with this
 * project's counter-based generator): with gamma = 0x9E3779B97F4A7C15 and
 * SplitMix64(z) the generator's output for state z + gamma, the stream state
 * is k = SplitMix64(seed) and entry i = BoxMuller(SplitMix64(k + 2i gamma),
 * SplitMix64(k + (2i+1) gamma)), uniforms (top 53 bits + 1) / 2^53;
 * unnormalised, written to the device array out [dim] of dtype (XD_C128:
 * real parts, zero imaginary parts).  Nearby seeds give independent vectors.
 * Asynchronous. */
xd_status xd_random_vector(int64_t dim, uint64_t seed, void *out,
                           xd_dtype dtype, xd_stream stream);

/* ---------------------------------------------------------------- batched */

/* ys[k] = H_k xs[k] for ninst independent U(1) Hamiltonians of uneven size
 * in one persistent launch (the multi-vector apply of Sec. 5.1 over many
 * blocks).  xs, ys: host arrays of ninst device pointers, each [dim_k][nvec]
 * (16-byte aligned for the eight-vector block product), x != y; dtype
 * XD_F32 or XD_F64; nvec in {1, 2, 4, 8}.  With eight FP32 right-hand sides
 * the operators large enough for the prefix-block layout (N >= 24, up to
 * 96 of them) are done inside the same launch by the eight-vector block
 * product.  The tile schedule is chosen by the library's autotuner (median
 * of five timings per candidate) on first use of a (set, dtype, nvec, stream)
 * and the launch is replayed from a captured CUDA graph while the pointers
 * are unchanged; new couplings of a member (xd_ham_set_couplings) or its
 * destruction drop the captured launch.  Errors: XD_EINVAL (NULL arrays or
 * vectors, x == y, a symmetric block, dtype or nvec), XD_ERANGE (more than
 * 512 bonds in an instance).  Asynchronous. */
xd_status xd_batch_apply(int ninst, const xd_ham *hs, const void *const *xs,
                         void *const *ys, xd_dtype dtype, int nvec,
                         xd_stream stream);

/* Thread-local description of the last error (never NULL). */
const char *xd_last_error(void);

/* Library version string. */
const char *xd_version(void);

/* Failure injection for testing error paths on the host: with n >= 0 the
 * library's next n device allocations succeed and the one after fails as an
 * out-of-memory error (the call that made it returns XD_ENOMEM, releasing
 * what it had allocated); the injection then switches itself off.  n < 0
 * switches it off at once.  Process-wide; always returns XD_OK. */
xd_status xd_debug_fail_alloc(int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* XDIAG_GPU_H */

/*
 * xd_oracle.c -- CPU oracle for the matrix-free spin-1/2 Heisenberg product.
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never links, loads or calls
 * this file; only tests/, __graft_entry__.smoke() and the CPU-baseline leg
 * of bench.py do.  It is plain, slow and written to be checked by eye
 * against the paper, in FP64 throughout.  It shares no code with the CUDA
 * library.
 *
 * Conventions (the paper's C++ reading, Sec. 3.1 and Sec. 3.10):
 *   - bit i of a state word is site i, a set bit is an up spin;
 *   - the U(1) block (N, nup) lists every N-bit word with nup set bits in
 *     ascending integer order, indices are 0-based;
 *   - H = sum_b J_b S_i.S_j with S = sigma/2 (Eq. 1, the SdotS type of
 *     App. A), S_i.S_j = Sz_i Sz_j + (S+_i S-_j + S-_i S+_j)/2: a bond with
 *     equal spins contributes +J/4 on the diagonal, a bond with opposite
 *     spins contributes -J/4 on the diagonal and J/2 to the state with both
 *     spins flipped (the Exchange type of Sec. 3.3 with real J).
 *   - a permutation g acts on a product state by (g s)_i = s_{g(i)}
 *     (Sec. 3.10); the symmetric state of a representative r is
 *     |r_chi> = (1/N_r) sum_g conj(chi(g)) g|r> (Sec. 3.10), the
 *     representative is the smallest integer of the orbit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "xd_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads used by the OpenMP loops below (always 1 without OpenMP); n >= 1
 * sets it.  Returns the count in force afterwards. */
int xo_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------- basics */

int64_t xo_binom(int n, int k)
{
    /* Pascal's rule, row by row; exact for n <= 64 (C(64,32) < 2^63). */
    if (k < 0 || n < 0 || k > n) return 0;
    int64_t row[65];
    for (int i = 0; i <= n; ++i) {
        row[i] = 1;
        for (int j = i - 1; j > 0; --j) row[j] = row[j] + row[j - 1];
    }
    return row[k];
}

int xo_popcount(uint64_t s)
{
    int c = 0;
    while (s) { c += (int)(s & 1u); s >>= 1; }
    return c;
}

static int bit(uint64_t s, int i) { return (int)((s >> i) & 1u); }

/* ------------------------------------------------------------ U(1) basis */

/* Every N-bit word with nup set bits, ascending (Sec. 3.1): scan all 2^N
 * words and keep those with the right popcount.  Returns the count; with
 * out == NULL only counts.  N <= 40 (the scan is 2^N steps). */
int64_t xo_enumerate(int N, int nup, uint64_t *out)
{
    if (N < 1 || N > 40 || nup < 0 || nup > N) return -1;
    int64_t n = 0;
    uint64_t end = (uint64_t)1 << N;
    for (uint64_t s = 0; s < end; ++s)
        if (xo_popcount(s) == nup) {
            if (out) out[n] = s;
            ++n;
        }
    return n;
}

/* Position of s in an ascending list (binary search), -1 if absent. */
int64_t xo_index_search(const uint64_t *states, int64_t dim, uint64_t s)
{
    int64_t lo = 0, hi = dim - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (states[mid] == s) return mid;
        if (states[mid] < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Position of s without the list: the number of words w < s with the same
 * popcount.  At the highest bit p where such a w differs from s, s has a 1
 * and w a 0, and w places the remaining ones freely in the p lower bits. */
int64_t xo_index_count(int N, int nup, uint64_t s)
{
    if (N < 64 && (s >> N)) return -1;
    if (xo_popcount(s) != nup) return -1;
    int64_t idx = 0;
    int ones = nup;
    for (int p = N - 1; p >= 0; --p)
        if (bit(s, p)) { idx += xo_binom(p, ones); --ones; }
    return idx;
}

/* Inverse of xo_index_count: the idx-th word (0-based) of the block. */
uint64_t xo_state_count(int N, int nup, int64_t idx)
{
    uint64_t s = 0;
    int ones = nup;
    for (int p = N - 1; p >= 0 && ones > 0; --p) {
        int64_t below = xo_binom(p, ones); /* words with a 0 at p */
        if (idx >= below) { s |= (uint64_t)1 << p; idx -= below; --ones; }
    }
    return s;
}

/* ------------------------------------------------------- random vectors */

/* One step of SplitMix64 (Steele, Lea, Flood 2014) from state z: the output
 * of the generator whose state is advanced from z to z + gamma. */
uint64_t xo_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Standard normal entry i of the seeded vector: Box-Muller on two uniforms
 * u = (top 53 bits + 1) / 2^53 in (0,1].  The seed is first mixed into a
 * stream state k = splitmix64(seed); entry i then takes outputs 2i+1 and
 * 2i+2 of the SplitMix64 stream started at k, i.e. splitmix64(k + 2i*gamma)
 * and splitmix64(k + (2i+1)*gamma), gamma = 0x9E3779B97F4A7C15.  Mixing the
 * seed makes the vectors of nearby seeds (seed, seed + 1, ...) independent
 * draws instead of permutations of one another.  (The paper draws N(0,1)
 * entries, Sec. 3.5; the generator itself is this project's choice.) */
double xo_rng_normal(uint64_t seed, int64_t i)
{
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    uint64_t k = xo_splitmix64(seed);
    uint64_t a = xo_splitmix64(k + (2u * (uint64_t)i) * gamma);
    uint64_t b = xo_splitmix64(k + (2u * (uint64_t)i + 1u) * gamma);
    double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;
    double u2 = ((double)(b >> 11) + 1.0) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

void xo_rng_fill(uint64_t seed, int64_t first, int64_t n, double *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = xo_rng_normal(seed, first + i);
}

/* Value keyed on a state word w (for vectors of blocks too large to list):
 * with k = splitmix64(seed), part 0 (real) and part 1 (imaginary) are
 *   2 u - 1,  u = (splitmix64(k + (2w + part) gamma) >> 11) 2^-53,
 * uniform in [-1, 1) and exactly representable, so any two implementations
 * of this definition give identical values. */
double xo_keyed(uint64_t seed, uint64_t w, int part)
{
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    uint64_t k = xo_splitmix64(seed);
    uint64_t z = xo_splitmix64(k + (2u * w + (uint64_t)part) * gamma);
    return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

/* ------------------------------------------------------------ H x (U(1)) */

/* y = H x on the U(1) block, pull form: row r of H applied to x (Eq. 1 with
 * the SdotS decomposition above).  x, y are row-major [dim][nvec]. */
void xo_apply_u1(int N, const uint64_t *states, int64_t dim, int nb,
                 const int32_t *bonds, const double *J, int nvec,
                 const double *x, double *y)
{
    (void)N;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t r = 0; r < dim; ++r) {
        uint64_t s = states[r];
        for (int v = 0; v < nvec; ++v) y[r * nvec + v] = 0.0;
        for (int b = 0; b < nb; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (bit(s, i) == bit(s, j)) {
                for (int v = 0; v < nvec; ++v)
                    y[r * nvec + v] += 0.25 * J[b] * x[r * nvec + v];
            } else {
                uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                int64_t c = xo_index_search(states, dim, t);
                for (int v = 0; v < nvec; ++v)
                    y[r * nvec + v] += -0.25 * J[b] * x[r * nvec + v]
                                       + 0.5 * J[b] * x[c * nvec + v];
            }
        }
    }
}

/* Selected rows of H x where x is the seeded normal vector (unnormalised),
 * using only the counting index: no list is stored, so this works at any
 * size.  rows[k] -> y[k]. */
void xo_apply_rows_rng(int N, int nup, int nb, const int32_t *bonds,
                       const double *J, uint64_t seed, const int64_t *rows,
                       int64_t nrows, double *y)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t r = rows[k];
        uint64_t s = xo_state_count(N, nup, r);
        double xr = xo_rng_normal(seed, r), acc = 0.0;
        for (int b = 0; b < nb; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (bit(s, i) == bit(s, j)) {
                acc += 0.25 * J[b] * xr;
            } else {
                uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                int64_t c = xo_index_count(N, nup, t);
                acc += -0.25 * J[b] * xr + 0.5 * J[b] * xo_rng_normal(seed, c);
            }
        }
        y[k] = acc;
    }
}

/* Flip targets of selected rows: for row r and bond b, the index of the
 * state with both spins of b flipped, or -1 when the spins are equal.
 * out is [nrows][nb]. */
void xo_flip_index_rows(int N, int nup, int nb, const int32_t *bonds,
                        const int64_t *rows, int64_t nrows, int64_t *out)
{
    for (int64_t k = 0; k < nrows; ++k) {
        uint64_t s = xo_state_count(N, nup, rows[k]);
        for (int b = 0; b < nb; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (bit(s, i) == bit(s, j)) { out[k * nb + b] = -1; continue; }
            uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
            out[k * nb + b] = xo_index_count(N, nup, t);
        }
    }
}

/* Per-bond bilinear forms out[b] = <g| S_i.S_j |x> (one term of H with unit
 * coupling), the derivative of <g|H|x> with respect to J_b. */
void xo_bond_forms(int N, const uint64_t *states, int64_t dim, int nb,
                   const int32_t *bonds, const double *g, const double *x,
                   double *out)
{
    (void)N;
    for (int b = 0; b < nb; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        double acc = 0.0;
        for (int64_t r = 0; r < dim; ++r) {
            uint64_t s = states[r];
            if (bit(s, i) == bit(s, j)) {
                acc += g[r] * 0.25 * x[r];
            } else {
                uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                int64_t c = xo_index_search(states, dim, t);
                acc += g[r] * (-0.25 * x[r] + 0.5 * x[c]);
            }
        }
        out[b] = acc;
    }
}

/* Two-point spin correlations <psi| O_ij |psi> of a U(1) state (the inner
 * product of Sec. 3.7 with the SzSz and SdotS operators of App. A on any site
 * pair).  kind 0: O = Sz_i Sz_j, +1/4 for equal spins and -1/4 for opposite
 * ones; kind 1: O = S_i.S_j, which adds (S+_i S-_j + S-_i S+_j)/2, taking a
 * state with opposite spins to the one with both flipped.  For i = j the
 * operators are (Sz_i)^2 = 1/4 and S_i.S_i = 3/4 (S(S+1) with S = 1/2). */
void xo_correlations(int N, const uint64_t *states, int64_t dim, int npairs,
                     const int32_t *pairs, int kind, const double *psi,
                     double *out)
{
    (void)N;
    for (int p = 0; p < npairs; ++p) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double acc = 0.0;
        for (int64_t r = 0; r < dim; ++r) {
            uint64_t s = states[r];
            double w = psi[r] * psi[r];
            if (i == j) {
                acc += (kind ? 0.75 : 0.25) * w;
            } else if (bit(s, i) == bit(s, j)) {
                acc += 0.25 * w;
            } else {
                acc -= 0.25 * w;
                if (kind) {
                    uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                    acc += 0.5 * psi[r] * psi[xo_index_search(states, dim, t)];
                }
            }
        }
        out[p] = acc;
    }
}

/* ------------------------------------------------------------- symmetry */

/* (g s)_i = s_{g(i)} (Sec. 3.10). */
uint64_t xo_act(int N, const int32_t *perm, uint64_t s)
{
    uint64_t t = 0;
    for (int i = 0; i < N; ++i)
        if (bit(s, perm[i])) t |= (uint64_t)1 << i;
    return t;
}

static int perm_equal(int N, const int32_t *a, const int32_t *b)
{
    for (int i = 0; i < N; ++i) if (a[i] != b[i]) return 0;
    return 1;
}

static int find_perm(int N, int G, const int32_t *perms, const int32_t *p)
{
    for (int g = 0; g < G; ++g) if (perm_equal(N, perms + (int64_t)g * N, p)) return g;
    return -1;
}

/* Group axioms (Sec. 3.9.1) and the homomorphism property of a 1-D
 * representation (Sec. 3.9.2).  Returns 0 when valid, else:
 * 1 a row is not a permutation, 2 no identity, 3 not closed under
 * composition, 4 an inverse is missing, 5 chi is not a homomorphism,
 * 6 |chi| != 1. */
int xo_group_check(int N, int G, const int32_t *perms, const double *chi_re,
                   const double *chi_im)
{
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int rc = 0, has_id = 0;
    for (int g = 0; g < G && !rc; ++g) {
        const int32_t *p = perms + (int64_t)g * N;
        memset(tmp, 0, sizeof(int32_t) * (size_t)N);
        int id = 1;
        for (int i = 0; i < N; ++i) {
            if (p[i] < 0 || p[i] >= N || tmp[p[i]]) { rc = 1; break; }
            tmp[p[i]] = 1;
            if (p[i] != i) id = 0;
        }
        if (!rc && id) has_id = 1;
    }
    if (!rc && !has_id) rc = 2;
    for (int f = 0; f < G && !rc; ++f)
        for (int g = 0; g < G && !rc; ++g) {
            const int32_t *pf = perms + (int64_t)f * N, *pg = perms + (int64_t)g * N;
            for (int i = 0; i < N; ++i) tmp[i] = pf[pg[i]]; /* f after g */
            int h = find_perm(N, G, perms, tmp);
            if (h < 0) { rc = 3; break; }
            if (chi_re) {
                double pr = chi_re[f] * chi_re[g] - chi_im[f] * chi_im[g];
                double pi = chi_re[f] * chi_im[g] + chi_im[f] * chi_re[g];
                if (fabs(pr - chi_re[h]) > 1e-9 || fabs(pi - chi_im[h]) > 1e-9) rc = 5;
            }
        }
    for (int g = 0; g < G && !rc; ++g) {
        const int32_t *p = perms + (int64_t)g * N;
        for (int i = 0; i < N; ++i) tmp[p[i]] = i;
        if (find_perm(N, G, perms, tmp) < 0) rc = 4;
        if (chi_re && fabs(hypot(chi_re[g], chi_im[g]) - 1.0) > 1e-9) rc = 6;
    }
    free(tmp);
    return rc;
}

/* Representative (smallest integer of the orbit, Sec. 3.10), the element
 * u with u s = rep (the first such g), and the number of g with g s = rep. */
uint64_t xo_rep(int N, int G, const int32_t *perms, uint64_t s, int *u,
                int *count)
{
    uint64_t best = ~(uint64_t)0;
    int bu = -1, cnt = 0;
    for (int g = 0; g < G; ++g) {
        uint64_t t = xo_act(N, perms + (int64_t)g * N, s);
        if (t < best) { best = t; bu = g; cnt = 1; }
        else if (t == best) ++cnt;
    }
    if (u) *u = bu;
    if (count) *count = cnt;
    return best;
}

/* Symmetry-adapted basis: the representatives r of the U(1) block whose
 * projected state does not vanish, i.e. sum_{g in Stab(r)} chi(g) != 0
 * (the norm N_r of Sec. 3.10 is then sqrt(|G| |Stab(r)|)).  Ascending.
 * Writes reps and |Stab(r)|; returns the count (out arrays may be NULL). */
int64_t xo_sym_basis(int N, int nup, int G, const int32_t *perms,
                     const double *chi_re, const double *chi_im,
                     uint64_t *reps, int32_t *stab)
{
    int64_t dim = xo_binom(N, nup), n = 0;
    for (int64_t k = 0; k < dim; ++k) {
        uint64_t s = xo_state_count(N, nup, k);
        int cnt;
        uint64_t r = xo_rep(N, G, perms, s, NULL, &cnt);
        if (r != s) continue;
        double sr = 0.0, si = 0.0;
        for (int g = 0; g < G; ++g)
            if (xo_act(N, perms + (int64_t)g * N, s) == s) { sr += chi_re[g]; si += chi_im[g]; }
        if (hypot(sr, si) < 1e-6) continue;
        if (reps) reps[n] = s;
        if (stab) stab[n] = cnt;
        ++n;
    }
    return n;
}

/* y = H x on the symmetry-adapted block, complex, pull form.  With
 * H|r> = sum_t h_t |s_t> and u_t s_t = r'_t:
 *   <r'_chi| H |r_chi> = sum_{t: r'_t = r'} h_t conj(chi(u_t)) N_{r'} / N_r,
 * so row r of H (Hermitian) is y_r = sum_t h_t chi(u_t) N_{r'_t}/N_r x_{r'_t}
 * with N_r = sqrt(|G| |Stab(r)|).  A target whose representative is not
 * in the block has a vanishing projection and contributes nothing.
 * x and y are interleaved complex [dim][2]. */
void xo_sym_apply(int N, int G, const int32_t *perms, const double *chi_re,
                  const double *chi_im, int nb, const int32_t *bonds,
                  const double *J, const uint64_t *reps, const int32_t *stab,
                  int64_t dim, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < dim; ++r) {
        uint64_t s = reps[r];
        double yr = 0.0, yi = 0.0, diag = 0.0;
        for (int b = 0; b < nb; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (bit(s, i) == bit(s, j)) { diag += 0.25 * J[b]; continue; }
            diag -= 0.25 * J[b];
            uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
            int u, cnt;
            uint64_t rp = xo_rep(N, G, perms, t, &u, &cnt);
            int64_t c = xo_index_search(reps, dim, rp);
            if (c < 0) continue;
            double amp = 0.5 * J[b] * sqrt((double)stab[c] / (double)stab[r]);
            double cr = amp * chi_re[u], ci = amp * chi_im[u];
            yr += cr * x[2 * c] - ci * x[2 * c + 1];
            yi += cr * x[2 * c + 1] + ci * x[2 * c];
        }
        y[2 * r] = yr + diag * x[2 * r];
        y[2 * r + 1] = yi + diag * x[2 * r + 1];
    }
}

/* Rows of y = H x on a symmetry-adapted block for a vector given by the keyed
 * values (x of the representative r is xo_keyed(seed, r, 0) + i
 * xo_keyed(seed, r, 1), real blocks: imaginary part 0).  For each requested
 * representative s (which must belong to the block) the row is the pull-form
 * row of xo_sym_apply, y_s = d(s) x_s + sum_t h_t chi(u_t) sqrt(|Stab(r'_t)| /
 * |Stab(s)|) x_{r'_t}, with the lookup of r'_t in a list of representatives
 * replaced by its membership test (sum_{g in Stab(r')} chi(g) != 0) and its
 * keyed value.  Lets sampled rows of blocks too large to enumerate be
 * checked.  y is interleaved complex [nrows][2]. */
void xo_sym_apply_rows_keyed(int N, int G, const int32_t *perms, const double *chi_re,
                             const double *chi_im, int nb, const int32_t *bonds,
                             const double *J, uint64_t seed, int cplx,
                             const uint64_t *rows, int64_t nrows, double *y)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nrows; ++q) {
        uint64_t s = rows[q];
        int cs;
        xo_rep(N, G, perms, s, NULL, &cs);
        double yr = 0.0, yi = 0.0, diag = 0.0;
        for (int b = 0; b < nb; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            if (bit(s, i) == bit(s, j)) { diag += 0.25 * J[b]; continue; }
            diag -= 0.25 * J[b];
            uint64_t t = s ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
            int u, cnt;
            uint64_t rp = xo_rep(N, G, perms, t, &u, &cnt);
            double sr = 0.0, si = 0.0;
            for (int g = 0; g < G; ++g)
                if (xo_act(N, perms + (int64_t)g * N, rp) == rp) { sr += chi_re[g]; si += chi_im[g]; }
            if (hypot(sr, si) < 1e-6) continue;
            double xr = xo_keyed(seed, rp, 0), xi = cplx ? xo_keyed(seed, rp, 1) : 0.0;
            double amp = 0.5 * J[b] * sqrt((double)cnt / (double)cs);
            double cr = amp * chi_re[u], ci = amp * chi_im[u];
            yr += cr * xr - ci * xi;
            yi += cr * xi + ci * xr;
        }
        double xr = xo_keyed(seed, s, 0), xi = cplx ? xo_keyed(seed, s, 1) : 0.0;
        y[2 * q] = yr + diag * xr;
        y[2 * q + 1] = yi + diag * xi;
    }
}

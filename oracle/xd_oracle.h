/* xd_oracle.h -- CPU oracle (test infrastructure only; see xd_oracle.c). */
#ifndef XD_ORACLE_H
#define XD_ORACLE_H
#include <stdint.h>

int xo_threads(int n);
int64_t xo_binom(int n, int k);
int xo_popcount(uint64_t s);
int64_t xo_enumerate(int N, int nup, uint64_t *out);
int64_t xo_index_search(const uint64_t *states, int64_t dim, uint64_t s);
int64_t xo_index_count(int N, int nup, uint64_t s);
uint64_t xo_state_count(int N, int nup, int64_t idx);
uint64_t xo_splitmix64(uint64_t z);
double xo_rng_normal(uint64_t seed, int64_t i);
void xo_rng_fill(uint64_t seed, int64_t first, int64_t n, double *out);
double xo_keyed(uint64_t seed, uint64_t w, int part);
void xo_apply_u1(int N, const uint64_t *states, int64_t dim, int nb,
                 const int32_t *bonds, const double *J, int nvec,
                 const double *x, double *y);
void xo_apply_rows_rng(int N, int nup, int nb, const int32_t *bonds,
                       const double *J, uint64_t seed, const int64_t *rows,
                       int64_t nrows, double *y);
void xo_flip_index_rows(int N, int nup, int nb, const int32_t *bonds,
                        const int64_t *rows, int64_t nrows, int64_t *out);
void xo_bond_forms(int N, const uint64_t *states, int64_t dim, int nb,
                   const int32_t *bonds, const double *g, const double *x,
                   double *out);
void xo_correlations(int N, const uint64_t *states, int64_t dim, int npairs,
                     const int32_t *pairs, int kind, const double *psi,
                     double *out);
uint64_t xo_act(int N, const int32_t *perm, uint64_t s);
int xo_group_check(int N, int G, const int32_t *perms, const double *chi_re,
                   const double *chi_im);
uint64_t xo_rep(int N, int G, const int32_t *perms, uint64_t s, int *u,
                int *count);
int64_t xo_sym_basis(int N, int nup, int G, const int32_t *perms,
                     const double *chi_re, const double *chi_im,
                     uint64_t *reps, int32_t *stab);
void xo_sym_apply(int N, int G, const int32_t *perms, const double *chi_re,
                  const double *chi_im, int nb, const int32_t *bonds,
                  const double *J, const uint64_t *reps, const int32_t *stab,
                  int64_t dim, const double *x, double *y);
void xo_sym_apply_rows_keyed(int N, int G, const int32_t *perms, const double *chi_re,
                             const double *chi_im, int nb, const int32_t *bonds,
                             const double *J, uint64_t seed, int cplx,
                             const uint64_t *rows, int64_t nrows, double *y);
#endif

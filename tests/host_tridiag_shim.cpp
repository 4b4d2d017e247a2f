// C entry points over xd_tridiag.h for the CPU tests (no CUDA).
#include <vector>

#include "xd_tridiag.h"

extern "C" double shim_tridiag_eig(int n, const double *d, const double *e, int k) { return xd::tridiag_eig(n, d, e, k); }

extern "C" void shim_tridiag_vec(int n, const double *d, const double *e, double lam, double *z) {
    xd::tridiag_vec(n, d, e, lam, z);
}

extern "C" void shim_ritz(int n, const double *alpha, const double *beta, int nev, double *evals, double *resid) {
    xd::ritz(n, alpha, beta, nev, evals, resid, nullptr);
}

extern "C" void shim_jacobi(int n, const double *A, double *Q, double *w) {
    std::vector<double> a(A, A + (size_t)n * n), q, ww;
    xd::jacobi_eig(n, a, q, ww);
    for (size_t i = 0; i < q.size(); ++i) Q[i] = q[i];
    for (int i = 0; i < n; ++i) w[i] = ww[i];
}

extern "C" void shim_expm_e1(int m, const double *alpha, const double *beta, double zr, double zi, double *cre,
                             double *cim) {
    std::vector<double> r, i;
    xd::expm_tridiag_e1(m, alpha, beta, zr, zi, r, i);
    for (int k = 0; k < m; ++k) {
        cre[k] = r[k];
        cim[k] = i[k];
    }
}

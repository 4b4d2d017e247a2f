// xd_tridiag.h -- host-side FP64 linear algebra of the Lanczos method
// (Sec. 3.6): eigenpairs of the tridiagonal T_m (Sturm bisection and inverse
// iteration; cyclic Jacobi) and exp(-z T_m) e_1 for the time evolution.
// Plain C++ without CUDA, so that the CPU tests compile it alone.
#pragma once

#include <math.h>

#include <algorithm>
#include <vector>

namespace xd {

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x
// (Sturm sequence of the LDL^T pivots).
inline int sturm_count(int n, const double *d, const double *e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
        double e2 = i ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i ? e2 / q : 0.0);
        if (q == 0.0) q = -1e-300;  // treat an exact zero pivot as negative
        if (q < 0) ++cnt;
    }
    return cnt;
}

// k-th smallest eigenvalue (0-based) by bisection on the Sturm count.
inline double tridiag_eig(int n, const double *d, const double *e, int k) {
    double lo = d[0], hi = d[0];
    for (int i = 0; i < n; ++i) {
        double r = (i ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    double scale = std::max(fabs(lo), fabs(hi)) + 1e-300;
    lo -= 1e-12 * scale;
    hi += 1e-12 * scale;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(n, d, e, mid) > k) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Eigenvector of (d, e) for eigenvalue lam by inverse iteration on
// (T - mu I) z = b with a pivoted tridiagonal LU (three sweeps).
inline void tridiag_vec(int n, const double *d, const double *e, double lam, double *z) {
    if (n == 1) {
        z[0] = 1.0;
        return;
    }
    double norm = 0.0;
    for (int i = 0; i < n; ++i) norm = std::max(norm, fabs(d[i]) + (i ? fabs(e[i - 1]) : 0) + (i < n - 1 ? fabs(e[i]) : 0));
    const double mu = lam + 1e-14 * (norm + 1e-300);
    // banded LU with partial pivoting: row i has entries at columns i..i+2 after pivoting
    std::vector<double> u0(n), u1(n), u2(n), l(n);
    std::vector<char> swp(n, 0);
    // current row i: (a = diag, b = super), next row: (c = sub, dd = diag, ee = super)
    double a = d[0] - mu, b = n > 1 ? e[0] : 0.0;
    double b2 = 0.0;
    for (int i = 0; i < n - 1; ++i) {
        double c = e[i], dd = d[i + 1] - mu, ee = (i + 2 < n) ? e[i + 1] : 0.0;
        if (fabs(c) > fabs(a)) {  // swap rows i and i+1
            swp[i] = 1;
            u0[i] = c;
            u1[i] = dd;
            u2[i] = ee;
            double m = a / c;
            l[i] = m;
            a = b - m * dd;
            b = b2 - m * ee;
            b2 = 0.0;
        } else {
            swp[i] = 0;
            u0[i] = a;
            u1[i] = b;
            u2[i] = b2;
            double m = (a != 0.0) ? c / a : 0.0;
            l[i] = m;
            a = dd - m * b;
            b = ee - m * b2;
            b2 = 0.0;
        }
    }
    u0[n - 1] = (a != 0.0) ? a : 1e-300;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
    std::vector<double> rhs(n, 1.0);
    for (int sweep = 0; sweep < 3; ++sweep) {
        // forward: apply the row swaps and multipliers
        std::vector<double> y(rhs);
        for (int i = 0; i < n - 1; ++i) {
            if (swp[i]) std::swap(y[i], y[i + 1]);
            y[i + 1] -= l[i] * y[i];
        }
        // back substitution
        for (int i = n - 1; i >= 0; --i) {
            double s = y[i];
            if (i + 1 < n) s -= u1[i] * z[i + 1];
            if (i + 2 < n) s -= u2[i] * z[i + 2];
            double piv = u0[i] != 0.0 ? u0[i] : 1e-300;
            z[i] = s / piv;
        }
        double nz = 0.0;
        for (int i = 0; i < n; ++i) nz += z[i] * z[i];
        nz = sqrt(nz);
        for (int i = 0; i < n; ++i) {
            z[i] /= nz;
            rhs[i] = z[i];
        }
    }
    // fix the sign: first non-negligible component positive
    for (int i = 0; i < n; ++i)
        if (fabs(z[i]) > 1e-8) {
            if (z[i] < 0)
                for (int k = 0; k < n; ++k) z[k] = -z[k];
            break;
        }
}

inline void ritz(int n, const double *alpha, const double *beta, int nev, double *evals,
                 double *resid, std::vector<double> *z0) {
    std::vector<double> z(n);
    for (int j = 0; j < nev; ++j) {
        if (j >= n) {
            evals[j] = NAN;
            resid[j] = NAN;
            continue;
        }
        evals[j] = tridiag_eig(n, alpha, beta, j);
        tridiag_vec(n, alpha, beta, evals[j], z.data());
        resid[j] = fabs(beta[n - 1] * z[n - 1]);
        if (j == 0 && z0) *z0 = z;
    }
}

// Eigenpairs of a symmetric n x n matrix by cyclic Jacobi rotations (the
// Jacobi eigenvalue method): A is destroyed, Q[i*n + j] = component i of
// eigenvector j, w[j] its eigenvalue.
inline void jacobi_eig(int n, std::vector<double> &A, std::vector<double> &Q, std::vector<double> &w) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                // rotation angle that zeroes A[p][q]: tan(2 phi) = 2 apq / (aqq - app)
                const double th = (aqq - app) / (2.0 * apq);
                const double tn = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(tn * tn + 1.0), s = tn * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
                    Q[(size_t)k * n + p] = c * qkp - s * qkq;
                    Q[(size_t)k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// c = exp(-z T) e_1 for the tridiagonal T = tridiag(beta, alpha, beta) of
// size m: T = Q diag(w) Q^T, c_k = sum_j Q[k][j] exp(-z w_j) Q[0][j].
inline void expm_tridiag_e1(int m, const double *alpha, const double *beta, double zr, double zi,
                            std::vector<double> &cre, std::vector<double> &cim) {
    std::vector<double> A((size_t)m * m, 0.0), Q, w;
    for (int k = 0; k < m; ++k) {
        A[(size_t)k * m + k] = alpha[k];
        if (k + 1 < m) A[(size_t)k * m + k + 1] = A[(size_t)(k + 1) * m + k] = beta[k];
    }
    jacobi_eig(m, A, Q, w);
    // shift by the smallest eigenvalue against overflow of exp(-tau w)
    double wmin = w.empty() ? 0.0 : *std::min_element(w.begin(), w.end());
    if (zr <= 0.0) wmin = 0.0;
    cre.assign(m, 0.0);
    cim.assign(m, 0.0);
    for (int j = 0; j < m; ++j) {
        const double mag = exp(-zr * (w[j] - wmin)), ph = -zi * w[j];
        const double er = mag * cos(ph), ei = mag * sin(ph);
        const double q0 = Q[j];  // Q[0][j]
        for (int k = 0; k < m; ++k) {
            cre[k] += Q[(size_t)k * m + j] * q0 * er;
            cim[k] += Q[(size_t)k * m + j] * q0 * ei;
        }
    }
    if (zr > 0.0) {  // undo the shift: exp(-zr wmin) overall
        const double f = exp(-zr * wmin);
        for (int k = 0; k < m; ++k) {
            cre[k] *= f;
            cim[k] *= f;
        }
    }
}

}  // namespace xd

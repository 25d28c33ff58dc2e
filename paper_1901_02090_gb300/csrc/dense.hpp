// Small dense FP64 linear algebra for the host-side setup (row-major).
//
// Cholesky, LU with partial pivoting, Householder null-space bases, a cyclic
// Jacobi symmetric eigensolver and Sturm bisection for symmetric tridiagonal
// matrices.  Sizes here are those of one subdomain's interface (tens to a few
// hundred) or of one face (a few to ~100), so plain loops suffice.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <vector>

namespace bddc {

using Vec = std::vector<double>;

// In-place Cholesky A = L L^T of an n x n SPD matrix (lower triangle used,
// upper triangle zeroed).  Returns false if a pivot is not positive.
inline bool chol(int n, double* A) {
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double d = std::sqrt(s);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / d;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0.0;
    }
    return true;
}

// Solve L L^T X = B for nrhs columns of B (B is n x nrhs row-major).
inline void chol_solve(int n, const double* L, double* B, int nrhs) {
    for (int i = 0; i < n; ++i) {
        double* bi = B + (size_t)i * nrhs;
        for (int k = 0; k < i; ++k) {
            const double l = L[(size_t)i * n + k];
            if (l == 0.0) continue;
            const double* bk = B + (size_t)k * nrhs;
            for (int c = 0; c < nrhs; ++c) bi[c] -= l * bk[c];
        }
        const double d = 1.0 / L[(size_t)i * n + i];
        for (int c = 0; c < nrhs; ++c) bi[c] *= d;
    }
    for (int i = n - 1; i >= 0; --i) {
        double* bi = B + (size_t)i * nrhs;
        for (int k = i + 1; k < n; ++k) {
            const double l = L[(size_t)k * n + i];
            if (l == 0.0) continue;
            const double* bk = B + (size_t)k * nrhs;
            for (int c = 0; c < nrhs; ++c) bi[c] -= l * bk[c];
        }
        const double d = 1.0 / L[(size_t)i * n + i];
        for (int c = 0; c < nrhs; ++c) bi[c] *= d;
    }
}

// In-place LU with partial pivoting; piv[i] = row swapped with i at step i.
// Returns false on an exactly zero pivot.
inline bool lu(int n, double* A, std::vector<int>& piv) {
    piv.resize(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            const double v = std::fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        if (p != k)
            for (int c = 0; c < n; ++c) std::swap(A[(size_t)k * n + c], A[(size_t)p * n + c]);
        const double inv = 1.0 / A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double* ai = A + (size_t)i * n;
            const double l = ai[k] * inv;
            ai[k] = l;
            if (l == 0.0) continue;
            const double* ak = A + (size_t)k * n;
            for (int c = k + 1; c < n; ++c) ai[c] -= l * ak[c];
        }
    }
    return true;
}

// Solve with the LU factors for nrhs columns (B is n x nrhs row-major).
inline void lu_solve(int n, const double* LU, const std::vector<int>& piv, double* B, int nrhs) {
    for (int k = 0; k < n; ++k)
        if (piv[k] != k)
            for (int c = 0; c < nrhs; ++c) std::swap(B[(size_t)k * nrhs + c], B[(size_t)piv[k] * nrhs + c]);
    for (int i = 0; i < n; ++i) {
        double* bi = B + (size_t)i * nrhs;
        for (int k = 0; k < i; ++k) {
            const double l = LU[(size_t)i * n + k];
            if (l == 0.0) continue;
            const double* bk = B + (size_t)k * nrhs;
            for (int c = 0; c < nrhs; ++c) bi[c] -= l * bk[c];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double* bi = B + (size_t)i * nrhs;
        for (int k = i + 1; k < n; ++k) {
            const double u = LU[(size_t)i * n + k];
            if (u == 0.0) continue;
            const double* bk = B + (size_t)k * nrhs;
            for (int c = 0; c < nrhs; ++c) bi[c] -= u * bk[c];
        }
        const double d = 1.0 / LU[(size_t)i * n + i];
        for (int c = 0; c < nrhs; ++c) bi[c] *= d;
    }
}

// Inverse from the LU factors, X = A^{-1} (n x n row-major): the operations
// of lu_solve on the identity without the products with the structural zeros
// of P I.  With the right-hand sides taken in pivot order the forward sweep
// solves with an identity, so row k of L^{-1} has entries in its first k + 1
// columns only (n^3 / 6 multiply-adds instead of n^3 / 2); every entry gets
// the same sequence of operations, so the result is bitwise that of
// lu_solve.
inline void lu_inverse(int n, const double* LU, const std::vector<int>& piv, double* X) {
    std::vector<int> perm(n), pos(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) std::swap(perm[k], perm[piv[k]]);
    for (int i = 0; i < n; ++i) pos[perm[i]] = i;  // the row of P I holding column c's 1
    std::vector<double> W((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double* wi = W.data() + (size_t)i * n;
        wi[i] = 1.0;
        for (int k = 0; k < i; ++k) {
            const double l = LU[(size_t)i * n + k];
            if (l == 0.0) continue;
            const double* wk = W.data() + (size_t)k * n;
            for (int c = 0; c <= k; ++c) wi[c] -= l * wk[c];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double* wi = W.data() + (size_t)i * n;
        for (int k = i + 1; k < n; ++k) {
            const double u = LU[(size_t)i * n + k];
            if (u == 0.0) continue;
            const double* wk = W.data() + (size_t)k * n;
            for (int c = 0; c < n; ++c) wi[c] -= u * wk[c];
        }
        const double d = 1.0 / LU[(size_t)i * n + i];
        for (int c = 0; c < n; ++c) wi[c] *= d;
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) X[(size_t)r * n + c] = W[(size_t)r * n + pos[c]];
}

// Orthonormal basis of the orthogonal complement of the row space of the
// m x n matrix C (rows assumed linearly independent), by Householder QR of
// C^T.  Returns Z as n x (n - m) row-major.
inline Vec null_space(int m, int n, const double* C) {
    Vec Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    Vec R((size_t)n * m);  // C^T, n x m
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) R[(size_t)j * m + i] = C[(size_t)i * n + j];
    Vec v(n);
    for (int k = 0; k < m && k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < n; ++i) nrm += R[(size_t)i * m + k] * R[(size_t)i * m + k];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        const double x0 = R[(size_t)k * m + k];
        const double alpha = x0 > 0 ? -nrm : nrm;
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        v[k] = x0 - alpha;
        for (int i = k + 1; i < n; ++i) v[i] = R[(size_t)i * m + k];
        double vv = 0.0;
        for (int i = k; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        for (int c = k; c < m; ++c) {   // R <- H R
            double s = 0.0;
            for (int i = k; i < n; ++i) s += v[i] * R[(size_t)i * m + c];
            s *= beta;
            for (int i = k; i < n; ++i) R[(size_t)i * m + c] -= s * v[i];
        }
        for (int r = 0; r < n; ++r) {   // Q <- Q H
            double s = 0.0;
            for (int i = k; i < n; ++i) s += Q[(size_t)r * n + i] * v[i];
            s *= beta;
            for (int i = k; i < n; ++i) Q[(size_t)r * n + i] -= s * v[i];
        }
    }
    const int nz = n - m;
    Vec Z((size_t)n * std::max(nz, 0));
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < nz; ++c) Z[(size_t)r * nz + c] = Q[(size_t)r * n + m + c];
    return Z;
}

// Cyclic Jacobi eigensolver for a symmetric n x n matrix A (destroyed).
// Returns eigenvalues in w and eigenvectors as columns of V (n x n).
inline void jacobi_eigh(int n, double* A, double* w, double* V) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Number of eigenvalues < x of the symmetric tridiagonal (d, e) (Sturm count).
inline int sturm_count(int n, const double* d, const double* e2, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < n; ++i) {
        q = d[i] - x - (i > 0 ? e2[i - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest and largest eigenvalue of a symmetric tridiagonal matrix with
// diagonal d and off-diagonal e (length n-1), by bisection.
inline void tridiag_extremes(int n, const double* d, const double* e, double* lmin, double* lmax) {
    std::vector<double> e2(std::max(n - 1, 1));
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
        if (i + 1 < n) e2[i] = e[i] * e[i];
    }
    auto kth = [&](int k) {  // k-th smallest (0-based)
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (a + b);
            if (m == a || m == b) break;
            if (sturm_count(n, d, e2.data(), m) > k) b = m; else a = m;
        }
        return 0.5 * (a + b);
    };
    *lmin = kth(0);
    *lmax = kth(n - 1);
}

}  // namespace bddc

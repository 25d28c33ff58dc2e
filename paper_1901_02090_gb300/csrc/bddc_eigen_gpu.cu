// The adaptive face eigenproblems of Algorithm 3 (Sec. 4.1), batched on the
// GPU in FP64.
//
// For the shared face Gamma^{ij} of subdomains i and j the pair problem of
// eq. (eigenvalue-problem-local-matrix) is solved in face-reduced form (the
// same steps as adaptive_face in bddc_setup.cpp):
//   T_i = [(S^i)^{-1}]_{face,face},  G = sym(T_i) + sym(T_j),
//   S_F = w_j S^i_ff w_j + w_i S^j_ff w_i          (elementwise weights),
//   Z   = an orthonormal basis of the complement of the face's net-flux
//         rows c o w_j, c o w_i (Householder QR),
//   A_r = Z^T S_F Z,  B_r = Z^T G^{-1} Z,  M = L^{-1} A_r L^{-T} (B_r = L L^T),
//   eigenpairs of M by cyclic Jacobi; the k eigenvalues above tau give the
//   rows S_F Z L^{-T} y, and omega^{ij} is the largest eigenvalue left.
// Two kernels:
//   k_fe_inverse  one CTA per subdomain: (S^i)^{-1} in place by Gauss-Jordan
//                 elimination (S^i is SPD, so no pivoting), which turns the
//                 T blocks of all of a subdomain's faces into gathers;
//   k_fe_face     one warp per face: the O(f^3) dense steps above, on a
//                 per-face slice of global scratch, each element of a step
//                 on one lane in the order of the sequential loop (the
//                 results do not depend on the lane count).
// The host keeps the last step (orthonormalising the rows against the
// face's existing constraint rows) and everything around it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bddc_internal.hpp"

namespace bddc {
namespace {

constexpr int kFeThreads = 256;

struct FeView {
    // subdomains: S^{-1} in place of S (n x n row-major, symmetric), weights
    const int* n;
    const int64_t *o_S, *o_w;
    double* Sinv;
    const double* S;
    const double* w;
    int* sub_status;
    // faces
    int nface;
    const int *fi, *fj, *ff;
    const int64_t *o_f, *o_rows, *o_scr;
    const int *pi, *pj;
    const double* coef;
    double tau;
    double* scr;
    double* omega;
    int* nrows;
    double* rows;
    int* face_status;
};

// (S^i)^{-1} by Gauss-Jordan elimination in place: step k scales row k by
// 1/a_kk and eliminates column k from every other row; the inverse builds
// up in the eliminated columns.  A non-positive pivot marks S^i as not
// positive definite.
__global__ void __launch_bounds__(kFeThreads) k_fe_inverse(FeView v) {
    const int s = blockIdx.x;
    const int n = v.n[s];
    double* A = v.Sinv + v.o_S[s];
    __shared__ double rowk[1024];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double piv = A[(int64_t)k * n + k];
        if (!(piv > 0.0)) {
            if (threadIdx.x == 0) bad = 1;
            break;
        }
        const double inv = 1.0 / piv;
        // new pivot row: a_kj / a_kk (j != k), 1 / a_kk at k
        for (int j = threadIdx.x; j < n; j += blockDim.x) rowk[j] = (j == k) ? inv : A[(int64_t)k * n + j] * inv;
        __syncthreads();
        // every other row: a_ij -= a_ik * newrow_j (j != k), a warp per row
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = wid; i < n; i += kFeThreads / 32) {
            if (i == k) continue;
            double* ai = A + (int64_t)i * n;
            const double aik = ai[k];
            for (int j = lane; j < n; j += 32)
                if (j != k) ai[j] -= aik * rowk[j];
        }
        __syncthreads();
        // column k: a_ik = -a_ik / a_kk
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != k) A[(int64_t)i * n + k] = -A[(int64_t)i * n + k] * inv;
        for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)k * n + j] = rowk[j];
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) v.sub_status[s] = bad ? BDDC_E_SETUP : BDDC_OK;
}

// ---- dense FP64 routines of one warp (row-major) ------------------------------------
// One warp per face.  Every output element is computed by one lane with the
// operations in the order of a sequential loop over the element's terms, so
// the results do not depend on how the elements are spread over the lanes;
// __syncwarp separates dependent steps.  Branch conditions are computed by
// every lane from the same values, so the warp stays converged.

// A = L L^T in place (L in the lower triangle, zeros above); false when A
// is not positive definite
__device__ bool fw_chol(int n, double* A) {
    const int l = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        double s = A[(int64_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(int64_t)j * n + k] * A[(int64_t)j * n + k];
        if (!(s > 0.0)) return false;
        const double d = sqrt(s);
        __syncwarp();
        for (int i = j + 1 + l; i < n; i += 32) {
            double t = A[(int64_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(int64_t)i * n + k] * A[(int64_t)j * n + k];
            A[(int64_t)i * n + j] = t / d;
        }
        for (int k = j + 1 + l; k < n; k += 32) A[(int64_t)j * n + k] = 0.0;
        if (l == 0) A[(int64_t)j * n + j] = d;
        __syncwarp();
    }
    return true;
}

// B <- A^{-1} B with the Cholesky factor L (A = L L^T), B n x m; a lane per column
__device__ void fw_chol_solve(int n, const double* L, double* B, int m) {
    for (int c = threadIdx.x & 31; c < m; c += 32) {
        for (int i = 0; i < n; ++i) {
            double v = B[(int64_t)i * m + c];
            for (int k = 0; k < i; ++k) v -= L[(int64_t)i * n + k] * B[(int64_t)k * m + c];
            B[(int64_t)i * m + c] = v / L[(int64_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = B[(int64_t)i * m + c];
            for (int k = i + 1; k < n; ++k) v -= L[(int64_t)k * n + i] * B[(int64_t)k * m + c];
            B[(int64_t)i * m + c] = v / L[(int64_t)i * n + i];
        }
    }
    __syncwarp();
}

// cyclic Jacobi eigensolver of a symmetric n x n A (destroyed): eigenvalues
// in w, eigenvectors as the columns of V.  The rotations run in the cyclic
// order; each one updates its two columns, then its two rows, then V, with
// a lane per index k.
__device__ void fw_jacobi(int n, double* A, double* w, double* V) {
    const int l = threadIdx.x & 31;
    for (int q = l; q < n * n; q += 32) V[q] = (q / n == q % n) ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a = A[(int64_t)i * n + j] * A[(int64_t)i * n + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(int64_t)p * n + q];
                if (fabs(apq) < 1e-300) continue;
                const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                __syncwarp();
                for (int k = l; k < n; k += 32) {
                    const double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
                    A[(int64_t)k * n + p] = c * akp - s * akq;
                    A[(int64_t)k * n + q] = s * akp + c * akq;
                }
                __syncwarp();
                for (int k = l; k < n; k += 32) {
                    const double apk = A[(int64_t)p * n + k], aqk = A[(int64_t)q * n + k];
                    A[(int64_t)p * n + k] = c * apk - s * aqk;
                    A[(int64_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = l; k < n; k += 32) {
                    const double vkp = V[(int64_t)k * n + p], vkq = V[(int64_t)k * n + q];
                    V[(int64_t)k * n + p] = c * vkp - s * vkq;
                    V[(int64_t)k * n + q] = s * vkp + c * vkq;
                }
                __syncwarp();
            }
    }
    for (int i = l; i < n; i += 32) w[i] = A[(int64_t)i * n + i];
    __syncwarp();
}

// the face-reduced pair eigenproblem of one face (one warp)
__global__ void __launch_bounds__(kFeThreads) k_fe_face(FeView v) {
    const int t = blockIdx.x * (kFeThreads / 32) + (threadIdx.x >> 5);
    if (t >= v.nface) return;  // whole warp
    const int l = threadIdx.x & 31;
    const int si = v.fi[t], sj = v.fj[t], f = v.ff[t];
    const int ni = v.n[si], nj = v.n[sj];
    const int* pi = v.pi + v.o_f[t];
    const int* pj = v.pj + v.o_f[t];
    const double* cf = v.coef + v.o_f[t];
    const double *Ii = v.Sinv + v.o_S[si], *Ij = v.Sinv + v.o_S[sj];
    const double *Si = v.S + v.o_S[si], *Sj = v.S + v.o_S[sj];
    const double *wi = v.w + v.o_w[si], *wj = v.w + v.o_w[sj];
    double* out_rows = v.rows + v.o_rows[t];
    if (l == 0) {
        v.omega[t] = 0.0;
        v.nrows[t] = 0;
        v.face_status[t] = BDDC_OK;
    }
    // scratch slices (f x f unless noted)
    double* base = v.scr + v.o_scr[t];
    const int64_t ff = (int64_t)f * f;
    double *G = base, *SF = G + ff, *Q = SF + ff, *Lg = Q + ff, *GiZ = Lg + ff, *Ar = GiZ + ff, *Br = Ar + ff,
           *M = Br + ff, *V = M + ff, *Z = V + ff, *vec = Z + ff;  // vec: 6 f
    double *lam = vec, *cm = vec + f, *hv = vec + 3 * f, *eta = vec + 4 * f, *delta = vec + 5 * f;
    // G = sym(T_i) + sym(T_j), S_F = w_j S^i_ff w_j + w_i S^j_ff w_i
    for (int64_t e = l; e < ff; e += 32) {
        const int a = (int)(e / f), b = (int)(e % f);
        const double tia = Ii[(int64_t)pi[a] * ni + pi[b]], tib = Ii[(int64_t)pi[b] * ni + pi[a]];
        const double tja = Ij[(int64_t)pj[a] * nj + pj[b]], tjb = Ij[(int64_t)pj[b] * nj + pj[a]];
        G[e] = 0.5 * (tia + tib) + 0.5 * (tja + tjb);
        SF[e] = wj[pj[a]] * Si[(int64_t)pi[a] * ni + pi[b]] * wj[pj[b]] +
                wi[pi[a]] * Sj[(int64_t)pj[a] * nj + pj[b]] * wi[pi[b]];
    }
    // the face's net-flux rows on the jump, c o w_j and c o w_i, orthonormalised
    // (the second dropped when it is (nearly) parallel to the first): lane 0
    int r = 0;
    if (l == 0) {
        for (int pass = 0; pass < 2; ++pass) {
            double* row = cm + (int64_t)r * f;
            double n0 = 0.0;
            for (int q = 0; q < f; ++q) {
                row[q] = cf[q] * (pass == 0 ? wj[pj[q]] : wi[pi[q]]);
                n0 += row[q] * row[q];
            }
            n0 = sqrt(n0);
            for (int rep = 0; rep < 2; ++rep)
                for (int b = 0; b < r; ++b) {
                    double dot = 0.0;
                    for (int q = 0; q < f; ++q) dot += cm[(int64_t)b * f + q] * row[q];
                    for (int q = 0; q < f; ++q) row[q] -= dot * cm[(int64_t)b * f + q];
                }
            double nn = 0.0;
            for (int q = 0; q < f; ++q) nn += row[q] * row[q];
            nn = sqrt(nn);
            if (n0 > 0 && nn > 1e-10 * n0) {
                for (int q = 0; q < f; ++q) row[q] /= nn;
                ++r;
            }
        }
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    const int nz = f - r;
    if (nz <= 0) return;  // whole warp
    // Z: the last f - r columns of Q of the Householder QR of C^T (f x r)
    for (int64_t e = l; e < ff; e += 32) Q[e] = (e / f == e % f) ? 1.0 : 0.0;
    __syncwarp();
    // R = C^T kept in Lg (f x r)
    for (int e = l; e < r * f; e += 32) {
        const int i = e / f, j = e % f;
        Lg[(int64_t)j * r + i] = cm[(int64_t)i * f + j];
    }
    __syncwarp();
    for (int k = 0; k < r && k < f; ++k) {
        // the reflector and the update of R on lane 0; then Q's rows, a lane per row
        double beta = 0.0;
        if (l == 0) {
            double nrm = 0.0;
            for (int i = k; i < f; ++i) nrm += Lg[(int64_t)i * r + k] * Lg[(int64_t)i * r + k];
            nrm = sqrt(nrm);
            if (nrm != 0.0) {
                const double x0 = Lg[(int64_t)k * r + k];
                const double alpha = x0 > 0 ? -nrm : nrm;
                for (int i = 0; i < f; ++i) hv[i] = 0.0;
                hv[k] = x0 - alpha;
                for (int i = k + 1; i < f; ++i) hv[i] = Lg[(int64_t)i * r + k];
                double vv = 0.0;
                for (int i = k; i < f; ++i) vv += hv[i] * hv[i];
                if (vv != 0.0) {
                    beta = 2.0 / vv;
                    for (int c = k; c < r; ++c) {
                        double s = 0.0;
                        for (int i = k; i < f; ++i) s += hv[i] * Lg[(int64_t)i * r + c];
                        s *= beta;
                        for (int i = k; i < f; ++i) Lg[(int64_t)i * r + c] -= s * hv[i];
                    }
                }
            }
        }
        beta = __shfl_sync(0xffffffffu, beta, 0);
        __syncwarp();
        if (beta == 0.0) continue;  // a zero column or reflector: no update (whole warp)
        for (int rr = l; rr < f; rr += 32) {
            double s = 0.0;
            for (int i = k; i < f; ++i) s += Q[(int64_t)rr * f + i] * hv[i];
            s *= beta;
            for (int i = k; i < f; ++i) Q[(int64_t)rr * f + i] -= s * hv[i];
        }
        __syncwarp();
    }
    for (int e = l; e < f * nz; e += 32) {
        const int a = e / nz, c = e % nz;
        Z[e] = Q[(int64_t)a * f + r + c];
    }
    // A_r = Z^T S_F Z, B_r = Z^T G^{-1} Z
    for (int64_t q = l; q < ff; q += 32) Lg[q] = G[q];
    __syncwarp();
    if (!fw_chol(f, Lg)) return;  // omega 0, no rows: as on the host
    for (int64_t q = l; q < (int64_t)f * nz; q += 32) GiZ[q] = Z[q];
    __syncwarp();
    fw_chol_solve(f, Lg, GiZ, nz);
    double* SFZ = M;  // f x nz, until M is formed
    for (int e = l; e < f * nz; e += 32) {
        const int a = e / nz, c = e % nz;
        double acc = 0.0;
        for (int b = 0; b < f; ++b) acc += SF[(int64_t)a * f + b] * Z[(int64_t)b * nz + c];
        SFZ[e] = acc;
    }
    __syncwarp();
    for (int e = l; e < nz * nz; e += 32) {
        const int x = e / nz, y = e % nz;
        double sa = 0.0, sb = 0.0;
        for (int a = 0; a < f; ++a) {
            sa += Z[(int64_t)a * nz + x] * SFZ[(int64_t)a * nz + y];
            sb += Z[(int64_t)a * nz + x] * GiZ[(int64_t)a * nz + y];
        }
        Ar[e] = sa;
        Br[e] = sb;
    }
    __syncwarp();
    for (int e = l; e < nz * nz; e += 32) {
        const int x = e / nz, y = e % nz;
        if (y <= x) continue;
        const double b = 0.5 * (Br[(int64_t)x * nz + y] + Br[(int64_t)y * nz + x]);
        const double a = 0.5 * (Ar[(int64_t)x * nz + y] + Ar[(int64_t)y * nz + x]);
        Br[(int64_t)x * nz + y] = Br[(int64_t)y * nz + x] = b;
        Ar[(int64_t)x * nz + y] = Ar[(int64_t)y * nz + x] = a;
    }
    __syncwarp();
    if (!fw_chol(nz, Br)) return;
    // M = L^{-1} A_r L^{-T}: a lane per column, then a lane per row
    for (int64_t q = l; q < (int64_t)nz * nz; q += 32) M[q] = Ar[q];
    __syncwarp();
    for (int c = l; c < nz; c += 32)
        for (int i = 0; i < nz; ++i) {
            double x = M[(int64_t)i * nz + c];
            for (int k = 0; k < i; ++k) x -= Br[(int64_t)i * nz + k] * M[(int64_t)k * nz + c];
            M[(int64_t)i * nz + c] = x / Br[(int64_t)i * nz + i];
        }
    __syncwarp();
    for (int rr = l; rr < nz; rr += 32)
        for (int i = 0; i < nz; ++i) {
            double x = M[(int64_t)rr * nz + i];
            for (int k = 0; k < i; ++k) x -= Br[(int64_t)i * nz + k] * M[(int64_t)rr * nz + k];
            M[(int64_t)rr * nz + i] = x / Br[(int64_t)i * nz + i];
        }
    __syncwarp();
    for (int e = l; e < nz * nz; e += 32) {
        const int x = e / nz, y = e % nz;
        if (y <= x) continue;
        M[(int64_t)x * nz + y] = M[(int64_t)y * nz + x] = 0.5 * (M[(int64_t)x * nz + y] + M[(int64_t)y * nz + x]);
    }
    __syncwarp();
    fw_jacobi(nz, M, lam, V);
    // eigenvalues in descending order (selection: stable, ties by index), the
    // count above tau and omega: lane 0
    int* idx = reinterpret_cast<int*>(Ar);  // A_r is no longer needed
    int k = 0;
    if (l == 0) {
        for (int q = 0; q < nz; ++q) idx[q] = q;
        for (int a = 1; a < nz; ++a) {
            const int key = idx[a];
            int b = a - 1;
            while (b >= 0 && lam[idx[b]] < lam[key]) {
                idx[b + 1] = idx[b];
                --b;
            }
            idx[b + 1] = key;
        }
        if (v.tau > 0 && isfinite(v.tau))
            while (k < nz && lam[idx[k]] > v.tau) ++k;
        v.omega[t] = k < nz ? fmax(lam[idx[k]], 0.0) : 0.0;
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    __syncwarp();
    // rows S_F Z L^{-T} y for the k eigenvectors y above tau
    for (int e = 0; e < k; ++e) {
        const int col = idx[e];
        for (int q = l; q < nz; q += 32) eta[q] = V[(int64_t)q * nz + col];
        __syncwarp();
        if (l == 0)
            for (int i = nz - 1; i >= 0; --i) {
                double x = eta[i];
                for (int kk = i + 1; kk < nz; ++kk) x -= Br[(int64_t)kk * nz + i] * eta[kk];
                eta[i] = x / Br[(int64_t)i * nz + i];
            }
        __syncwarp();
        for (int a = l; a < f; a += 32) {
            double d = 0.0;
            for (int q = 0; q < nz; ++q) d += Z[(int64_t)a * nz + q] * eta[q];
            delta[a] = d;
        }
        __syncwarp();
        for (int a = l; a < f; a += 32) {
            double s = 0.0;
            for (int b = 0; b < f; ++b) s += SF[(int64_t)a * f + b] * delta[b];
            out_rows[(int64_t)e * f + a] = s;
        }
        __syncwarp();
    }
    if (l == 0) v.nrows[t] = k;
}

template <class T>
bool up(const std::vector<T>& h, T** d) {
    *d = nullptr;
    if (cudaMalloc((void**)d, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) return false;
    if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    return true;
}

}  // namespace

int face_eigen_device(FaceEigenBatch& B, std::string& err) {
    const int ns = (int)B.n.size(), nf = (int)B.ff.size();
    B.omega.assign(nf, 0.0);
    B.nrows.assign(nf, 0);
    B.rows.assign((size_t)B.o_rows.back(), 0.0);
    B.face_status.assign(nf, BDDC_OK);
    B.sub_status.assign(ns, BDDC_OK);
    if (nf == 0) return BDDC_OK;
    for (int s = 0; s < ns; ++s)
        if (B.n[s] > 1024) {
            err = "interface of more than 1024 dofs";
            return BDDC_E_INVALID_ARG;
        }
    std::vector<void*> owned;
    auto release = [&]() {
        for (void* p : owned) cudaFree(p);
        owned.clear();
    };
    int rc = BDDC_OK;
    auto track = [&](bool ok, void* p) {
        if (p) owned.push_back(p);
        if (!ok && !rc) rc = BDDC_E_OOM;
    };
    FeView v{};
    int *d_n = nullptr, *d_fi = nullptr, *d_fj = nullptr, *d_ff = nullptr, *d_pi = nullptr, *d_pj = nullptr;
    int64_t *d_oS = nullptr, *d_ow = nullptr, *d_of = nullptr, *d_orows = nullptr;
    double *d_S = nullptr, *d_Sinv = nullptr, *d_w = nullptr, *d_coef = nullptr;
    track(up(B.n, &d_n), d_n);
    track(up(B.o_S, &d_oS), d_oS);
    track(up(B.o_w, &d_ow), d_ow);
    track(up(B.S, &d_S), d_S);
    track(up(B.S, &d_Sinv), d_Sinv);
    track(up(B.w, &d_w), d_w);
    track(up(B.fi, &d_fi), d_fi);
    track(up(B.fj, &d_fj), d_fj);
    track(up(B.ff, &d_ff), d_ff);
    track(up(B.o_f, &d_of), d_of);
    track(up(B.o_rows, &d_orows), d_orows);
    track(up(B.pi, &d_pi), d_pi);
    track(up(B.pj, &d_pj), d_pj);
    track(up(B.coef, &d_coef), d_coef);
    // per-face scratch: 10 f x f slices and 6 f vectors, faces in chunks of <= 1 GB
    std::vector<int64_t> o_scr(nf + 1, 0);
    for (int t = 0; t < nf; ++t) o_scr[t + 1] = o_scr[t] + 10LL * B.ff[t] * B.ff[t] + 6LL * B.ff[t];
    double *d_omega = nullptr, *d_rows = nullptr;
    int *d_nrows = nullptr, *d_fst = nullptr, *d_sst = nullptr;
    track(cudaMalloc((void**)&d_omega, sizeof(double) * nf) == cudaSuccess, d_omega);
    track(cudaMalloc((void**)&d_nrows, sizeof(int) * nf) == cudaSuccess, d_nrows);
    track(cudaMalloc((void**)&d_fst, sizeof(int) * nf) == cudaSuccess, d_fst);
    track(cudaMalloc((void**)&d_sst, sizeof(int) * std::max(ns, 1)) == cudaSuccess, d_sst);
    track(cudaMalloc((void**)&d_rows, sizeof(double) * std::max<int64_t>(B.o_rows.back(), 1)) == cudaSuccess, d_rows);
    if (rc) {
        cudaGetLastError();
        release();
        err = "device memory for the face eigenproblems";
        return rc;
    }
    v.n = d_n;
    v.o_S = d_oS;
    v.o_w = d_ow;
    v.S = d_S;
    v.Sinv = d_Sinv;
    v.w = d_w;
    v.sub_status = d_sst;
    v.fi = d_fi;
    v.fj = d_fj;
    v.ff = d_ff;
    v.o_f = d_of;
    v.o_rows = d_orows;
    v.pi = d_pi;
    v.pj = d_pj;
    v.coef = d_coef;
    v.tau = B.tau;
    v.omega = d_omega;
    v.nrows = d_nrows;
    v.rows = d_rows;
    v.face_status = d_fst;
    k_fe_inverse<<<ns, kFeThreads>>>(v);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        release();
        err = "device inverse of the interface Schur complements";
        return BDDC_E_CUDA;
    }
    cudaMemcpy(B.sub_status.data(), d_sst, sizeof(int) * ns, cudaMemcpyDeviceToHost);
    for (int s = 0; s < ns; ++s)
        if (B.sub_status[s] != BDDC_OK) {
            release();
            err = "interface Schur complement not positive definite";
            return BDDC_E_SETUP;
        }
    const int64_t kChunkDoubles = (1LL << 30) / 8;
    double* d_scr = nullptr;
    int64_t cap = 0;
    for (int t0 = 0; t0 < nf;) {
        int t1 = t0 + 1;
        while (t1 < nf && o_scr[t1 + 1] - o_scr[t0] <= kChunkDoubles) ++t1;
        const int64_t need = o_scr[t1] - o_scr[t0];
        if (need > cap) {
            if (d_scr) cudaFree(d_scr);
            d_scr = nullptr;
            if (cudaMalloc((void**)&d_scr, sizeof(double) * need) != cudaSuccess) {
                cudaGetLastError();
                release();
                err = "device scratch for the face eigenproblems";
                return BDDC_E_OOM;
            }
            cap = need;
        }
        std::vector<int64_t> o_loc(t1 - t0);
        for (int t = t0; t < t1; ++t) o_loc[t - t0] = o_scr[t] - o_scr[t0];
        int64_t* d_oscr = nullptr;
        if (!up(o_loc, &d_oscr)) {
            cudaGetLastError();
            if (d_oscr) cudaFree(d_oscr);
            cudaFree(d_scr);
            release();
            err = "device memory for the face eigenproblems";
            return BDDC_E_OOM;
        }
        FeView c = v;
        c.nface = t1 - t0;
        c.fi = d_fi + t0;
        c.fj = d_fj + t0;
        c.ff = d_ff + t0;
        c.o_f = d_of + t0;
        c.o_rows = d_orows + t0;
        c.o_scr = d_oscr;
        c.scr = d_scr;
        c.omega = d_omega + t0;
        c.nrows = d_nrows + t0;
        c.face_status = d_fst + t0;
        k_fe_face<<<(c.nface + kFeThreads / 32 - 1) / (kFeThreads / 32), kFeThreads>>>(c);
        const cudaError_t e = cudaDeviceSynchronize();
        cudaFree(d_oscr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d_scr);
            release();
            err = "device face eigenproblems";
            return BDDC_E_CUDA;
        }
        t0 = t1;
    }
    if (d_scr) cudaFree(d_scr);
    bool ok = cudaMemcpy(B.omega.data(), d_omega, sizeof(double) * nf, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(B.nrows.data(), d_nrows, sizeof(int) * nf, cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaMemcpy(B.rows.data(), d_rows, sizeof(double) * B.rows.size(), cudaMemcpyDeviceToHost) == cudaSuccess;
    release();
    if (!ok) {
        cudaGetLastError();
        err = "copy of the face eigenproblem results";
        return BDDC_E_CUDA;
    }
    return BDDC_OK;
}

}  // namespace bddc

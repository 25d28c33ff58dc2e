// Dense part of the local maps of a batch of subdomains, on the GPU.
//
// For subdomain i the setup solves the interior problem of the local mixed
// system (interior fluxes, cell pressures, and the multiplier of the
// mean-pressure constraint) for every interface flux dof and every cell
// source: the columns give S^i (the flux Schur complement on the interface,
// Sec. 3), G_pre (Step 2) and G_post (the post-correction).  The interior
// block A_II is tridiagonal along grid lines ("chains", factored on the
// host); eliminating it leaves the dense pressure Schur complement
//     Q = [[-dB_I A_II^{-1} dB_I^T, v], [v^T, 0]]      (n_c + 1 square)
// which is LU-factored with partial pivoting.  All right-hand sides are
// solved together (the interior fluxes last, u = A_II^{-1}(x_u - dB_I^T p),
// two chain solves per column) and refined against the exact sparse local
// operator (the elimination loses accuracy in proportion to the
// permeability contrast).  This is the algorithm of local_maps in
// bddc_setup.cpp step by step (kLocalRefinements steps of refinement);
// here one CTA takes one subdomain and its threads take the
// right-hand-side columns, in FP64.
//
// Scratch layouts are column-fastest ([row * ncol + column]) so that the
// threads of a warp, one column each, touch consecutive addresses.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bddc_internal.hpp"

namespace bddc {
namespace {

constexpr double kMassDiagD = 1.0 / 3.0;  // RT0 mass block of a cell: (1/3, 1/6; 1/6, 1/3) per axis
constexpr double kMassOffD = 1.0 / 6.0;
constexpr int kLmThreads = 256;

struct LmView {
    int sub0;  // first subdomain (batch index) of this launch
    const int *dim, *ng, *ni, *nc;
    const double *vol, *d;
    const int64_t *o_cell, *o_ng, *o_ni, *o_ch, *o_S, *o_Gpre, *o_Gpost;
    const int *clo, *chi;
    const double* cs;
    const int *gcell, *gaxis, *gside;
    const int *order, *cstart;
    const double *rdfac, *lfac, *off;  // Thomas factors (rdfac: pivot reciprocals)
    double *S, *GpreT, *GpostT;
    int* status;
    // scratch, per launch-local subdomain t: offsets o_*[t]
    const int64_t *o_Y, *o_Q, *o_U, *o_P, *o_piv;
    double *Y, *Q, *XU, *YU, *RU, *DU, *XP, *YP, *RP, *DP;
    int* piv;
};

struct Dims {
    int s, t, dim, ng, ni, nc, nq, ncol;
    double vol, d;
};
__device__ __forceinline__ Dims dims(const LmView& v) {
    Dims q;
    q.t = blockIdx.x;
    q.s = v.sub0 + q.t;
    q.dim = v.dim[q.s];
    q.ng = v.ng[q.s];
    q.ni = v.ni[q.s];
    q.nc = v.nc[q.s];
    q.nq = q.nc + 1;
    q.ncol = q.ng + q.nc;
    q.vol = v.vol[q.s];
    q.d = v.d[q.s];
    return q;
}

// x <- A_II^{-1} x for an interior vector stored with stride `stride`
__device__ void chain_solve(const LmView& v, const Dims& q, double* x, int stride) {
    const int64_t ob = v.o_ni[q.s];
    const int* ord = v.order + ob;
    const double *lf = v.lfac + ob, *rd = v.rdfac + ob, *of = v.off + ob;
    for (int64_t c = v.o_ch[q.s]; c + 1 < v.o_ch[q.s + 1]; ++c) {
        const int b = v.cstart[c], e = v.cstart[c + 1];
        for (int p = b + 1; p < e; ++p) x[(int64_t)ord[p] * stride] -= lf[p] * x[(int64_t)ord[p - 1] * stride];
        x[(int64_t)ord[e - 1] * stride] *= rd[e - 1];
        for (int p = e - 2; p >= b; --p)
            x[(int64_t)ord[p] * stride] = (x[(int64_t)ord[p] * stride] - of[p] * x[(int64_t)ord[p + 1] * stride]) * rd[p];
    }
}

// (dB_I t)_r for the interior vector t (stride `stride`)
__device__ __forceinline__ double dBI_row(const LmView& v, const Dims& q, const double* t, int stride, int r) {
    const int64_t cb = (v.o_cell[q.s] + r) * 3;
    double val = 0.0;
    for (int a = 0; a < q.dim; ++a) {
        const int l = v.clo[cb + a], h = v.chi[cb + a];
        if (l >= q.ng) val += t[(int64_t)(l - q.ng) * stride];
        if (h >= q.ng) val -= t[(int64_t)(h - q.ng) * stride];
    }
    return q.d * val;
}

// Y = A_II^{-1} dB_I^T, column r per thread ([e * nc + r])
__global__ void __launch_bounds__(kLmThreads) k_lm_Y(LmView v) {
    const Dims q = dims(v);
    double* Y = v.Y + v.o_Y[q.t];
    for (int r = threadIdx.x; r < q.nc; r += blockDim.x) {
        for (int e = 0; e < q.ni; ++e) Y[(int64_t)e * q.nc + r] = 0.0;
        const int64_t cb = (v.o_cell[q.s] + r) * 3;
        for (int a = 0; a < q.dim; ++a) {
            const int l = v.clo[cb + a], h = v.chi[cb + a];
            if (l >= q.ng) Y[(int64_t)(l - q.ng) * q.nc + r] += q.d;  // B[c, lower] = +1
            if (h >= q.ng) Y[(int64_t)(h - q.ng) * q.nc + r] -= q.d;  // B[c, upper] = -1
        }
        chain_solve(v, q, Y + r, q.nc);
    }
}

// Q = [[-dB_I Y, v], [v^T, 0]] (row-major, nq x nq), column r per thread
__global__ void __launch_bounds__(kLmThreads) k_lm_Q(LmView v) {
    const Dims q = dims(v);
    const double* Y = v.Y + v.o_Y[q.t];
    double* Q = v.Q + v.o_Q[q.t];
    for (int r = threadIdx.x; r < q.nc; r += blockDim.x) {
        for (int rr = 0; rr < q.nc; ++rr) Q[(int64_t)rr * q.nq + r] = -dBI_row(v, q, Y + r, q.nc, rr);
        Q[(int64_t)r * q.nq + q.nc] = q.vol;
        Q[(int64_t)q.nc * q.nq + r] = q.vol;
    }
    if (threadIdx.x == 0) Q[(int64_t)q.nc * q.nq + q.nc] = 0.0;
}

// in-place LU of Q with partial pivoting (the pivot is the first row of
// largest magnitude in the column, as on the host); multipliers in the
// strict lower triangle, U above it with the reciprocals of its pivots on
// the diagonal, piv[k] the row swapped with k
__global__ void __launch_bounds__(kLmThreads) k_lm_lu(LmView v) {
    extern __shared__ double lcol[];  // multipliers of the current step
    __shared__ int piv_sh, bad_sh;
    const Dims q = dims(v);
    double* A = v.Q + v.o_Q[q.t];
    int* piv = v.piv + v.o_piv[q.t];
    const int n = q.nq;
    // identity first: a factorisation that stops early leaves valid indices
    for (int i = threadIdx.x; i < n; i += blockDim.x) piv[i] = i;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x < 32) {
            // lane-strided scan keeps the first strict maximum, then the
            // xor-combine prefers the larger value, the smaller row on ties
            double best = -1.0;
            int p = n;
            for (int i = k + (int)threadIdx.x; i < n; i += 32) {
                const double a = fabs(A[(int64_t)i * n + k]);
                if (a > best || (a != a && best == best)) {  // NaN wins so that it is reported
                    best = a;
                    p = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int op = __shfl_xor_sync(0xffffffffu, p, o);
                if (ob > best || (ob == best && op < p) || (ob != ob && best == best)) {
                    best = ob;
                    p = op;
                }
            }
            if (threadIdx.x == 0) {
                piv_sh = p;
                bad_sh = !(best > 0.0) || !isfinite(best);
            }
        }
        __syncthreads();
        const int p = piv_sh;
        if (bad_sh) {
            if (threadIdx.x == 0) v.status[q.s] = BDDC_E_SETUP;
            return;
        }
        if (threadIdx.x == 0) piv[k] = p;
        if (p != k)
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                const double t = A[(int64_t)k * n + c];
                A[(int64_t)k * n + c] = A[(int64_t)p * n + c];
                A[(int64_t)p * n + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / A[(int64_t)k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double l = A[(int64_t)i * n + k] * inv;
            A[(int64_t)i * n + k] = l;
            lcol[i] = l;
        }
        __syncthreads();
        for (int c = k + 1 + threadIdx.x; c < n; c += blockDim.x) {
            const double akc = A[(int64_t)k * n + c];
            for (int i = k + 1; i < n; ++i) {
                const double l = lcol[i];
                if (l != 0.0) A[(int64_t)i * n + c] -= l * akc;
            }
        }
        __syncthreads();
    }
    // the diagonal of U is kept as its reciprocals (the solves multiply)
    for (int i = threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + i] = 1.0 / A[(int64_t)i * n + i];
}

// right-hand sides: interface column j < ng is -K_I,G e_j (the other flux
// face of its cell along its axis, and -dB_G e_j on its cell's pressure);
// column ng + r is the unit source d |c_r| on cell r
__global__ void __launch_bounds__(kLmThreads) k_lm_rhs(LmView v) {
    const Dims q = dims(v);
    if (v.status[q.s] != BDDC_OK) return;  // singular pressure Schur complement
    double* XU = v.XU + v.o_U[q.t];
    double* XP = v.XP + v.o_P[q.t];
    for (int j = threadIdx.x; j < q.ncol; j += blockDim.x) {
        for (int e = 0; e < q.ni; ++e) XU[(int64_t)e * q.ncol + j] = 0.0;
        for (int r = 0; r < q.nq; ++r) XP[(int64_t)r * q.ncol + j] = 0.0;
        if (j < q.ng) {
            const int64_t gj = v.o_ng[q.s] + j;
            const int r = v.gcell[gj], a = v.gaxis[gj], side = v.gside[gj];
            const int64_t cb = (v.o_cell[q.s] + r) * 3;
            const double sc = v.cs[cb + a];
            const int other = side == 0 ? v.chi[cb + a] : v.clo[cb + a];
            if (other >= q.ng) XU[(int64_t)(other - q.ng) * q.ncol + j] = -kMassOffD * sc;
            XP[(int64_t)r * q.ncol + j] = -q.d * (side == 0 ? 1.0 : -1.0);
        } else {
            XP[(int64_t)(j - q.ng) * q.ncol + j] = -q.d * q.vol;
        }
    }
}

// solve K_I [yu; yp] = [xu; xp] for every column (one column per thread):
// interior elimination, LU solve of the pressure Schur complement, the
// interior fluxes from a second chain solve
__global__ void __launch_bounds__(kLmThreads) k_lm_solve(LmView v, const double* xu_all, const double* xp_all,
                                                          double* yu_all, double* yp_all) {
    const Dims q = dims(v);
    if (v.status[q.s] != BDDC_OK) return;  // singular pressure Schur complement
    const double* xu = xu_all + v.o_U[q.t];
    const double* xp = xp_all + v.o_P[q.t];
    double* yu = yu_all + v.o_U[q.t];
    double* yp = yp_all + v.o_P[q.t];
    const double* LU = v.Q + v.o_Q[q.t];
    const int* piv = v.piv + v.o_piv[q.t];
    const int n = q.nq, nc = q.ncol;
    for (int j = threadIdx.x; j < q.ncol; j += blockDim.x) {
        double* u = yu + j;
        double* pp = yp + j;
        for (int e = 0; e < q.ni; ++e) u[(int64_t)e * nc] = xu[(int64_t)e * nc + j];
        for (int r = 0; r < n; ++r) pp[(int64_t)r * nc] = xp[(int64_t)r * nc + j];
        chain_solve(v, q, u, nc);
        for (int r = 0; r < q.nc; ++r) pp[(int64_t)r * nc] -= dBI_row(v, q, u, nc, r);
        for (int k = 0; k < n; ++k)
            if (piv[k] != k) {
                const double t = pp[(int64_t)k * nc];
                pp[(int64_t)k * nc] = pp[(int64_t)piv[k] * nc];
                pp[(int64_t)piv[k] * nc] = t;
            }
        for (int i = 0; i < n; ++i) {
            double acc = pp[(int64_t)i * nc];
            for (int k = 0; k < i; ++k) {
                const double l = LU[(int64_t)i * n + k];
                if (l != 0.0) acc -= l * pp[(int64_t)k * nc];
            }
            pp[(int64_t)i * nc] = acc;
        }
        for (int i = n - 1; i >= 0; --i) {
            double acc = pp[(int64_t)i * nc];
            for (int k = i + 1; k < n; ++k) {
                const double uu = LU[(int64_t)i * n + k];
                if (uu != 0.0) acc -= uu * pp[(int64_t)k * nc];
            }
            pp[(int64_t)i * nc] = acc * LU[(int64_t)i * n + i];  // the stored reciprocal
        }
        // u = A_II^{-1} (x_u - dB_I^T y_p): the sparse transpose and a second
        // chain solve (n_i work per column) in place of the dense product
        // with Y (n_i n_c work per column)
        for (int e = 0; e < q.ni; ++e) u[(int64_t)e * nc] = xu[(int64_t)e * nc + j];
        const int64_t cb0 = v.o_cell[q.s] * 3;
        for (int r = 0; r < q.nc; ++r) {
            const double yr = pp[(int64_t)r * nc];
            if (yr == 0.0) continue;
            for (int a = 0; a < q.dim; ++a) {
                const int l = v.clo[cb0 + 3 * r + a], h = v.chi[cb0 + 3 * r + a];
                if (l >= q.ng) u[(int64_t)(l - q.ng) * nc] -= q.d * yr;  // B[c, lower] = +1
                if (h >= q.ng) u[(int64_t)(h - q.ng) * nc] += q.d * yr;  // B[c, upper] = -1
            }
        }
        chain_solve(v, q, u, nc);
    }
}

// residual [ru; rp] = [xu; xp] - K_I [yu; yp] against the exact sparse operator
__global__ void __launch_bounds__(kLmThreads) k_lm_resid(LmView v) {
    const Dims q = dims(v);
    if (v.status[q.s] != BDDC_OK) return;  // singular pressure Schur complement
    const double* XU = v.XU + v.o_U[q.t];
    const double* XP = v.XP + v.o_P[q.t];
    const double* YU = v.YU + v.o_U[q.t];
    const double* YP = v.YP + v.o_P[q.t];
    double* RU = v.RU + v.o_U[q.t];
    double* RP = v.RP + v.o_P[q.t];
    const int nc = q.ncol;
    for (int j = threadIdx.x; j < q.ncol; j += blockDim.x) {
        const double* yu = YU + j;
        double* ru = RU + j;
        for (int e = 0; e < q.ni; ++e) ru[(int64_t)e * nc] = XU[(int64_t)e * nc + j];
        const double ymu = YP[(int64_t)q.nc * nc + j];
        double sump = 0.0;
        for (int r = 0; r < q.nc; ++r) {
            const double y = YP[(int64_t)r * nc + j];
            sump += y;
            double divr = 0.0;
            const int64_t cb = (v.o_cell[q.s] + r) * 3;
            for (int a = 0; a < q.dim; ++a) {
                const double sc = v.cs[cb + a];
                const int l = v.clo[cb + a], h = v.chi[cb + a];
                const bool li = l >= q.ng, hi = h >= q.ng;
                const double vl = li ? yu[(int64_t)(l - q.ng) * nc] : 0.0;
                const double vh = hi ? yu[(int64_t)(h - q.ng) * nc] : 0.0;
                if (li) ru[(int64_t)(l - q.ng) * nc] -= kMassDiagD * sc * vl + kMassOffD * sc * vh + q.d * y;
                if (hi) ru[(int64_t)(h - q.ng) * nc] -= kMassOffD * sc * vl + kMassDiagD * sc * vh - q.d * y;
                divr += q.d * (vl - vh);
            }
            RP[(int64_t)r * nc + j] = XP[(int64_t)r * nc + j] - divr - q.vol * ymu;
        }
        RP[(int64_t)q.nc * nc + j] = XP[(int64_t)q.nc * nc + j] - q.vol * sump;
    }
}

__global__ void k_lm_add(int64_t n, double* y, const double* dy) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += dy[i];
}

// outputs per column j: G_post column (interior fluxes, pressures), and the
// interface residual, which is column j of S (j < ng) or of G_pre
__global__ void __launch_bounds__(kLmThreads) k_lm_out(LmView v) {
    const Dims q = dims(v);
    if (v.status[q.s] != BDDC_OK) return;  // singular pressure Schur complement
    const double* YU = v.YU + v.o_U[q.t];
    const double* YP = v.YP + v.o_P[q.t];
    const int nc = q.ncol;
    for (int j = threadIdx.x; j < q.ncol; j += blockDim.x) {
        double* post = v.GpostT + v.o_Gpost[q.s] + (int64_t)j * (q.ni + q.nc);
        for (int e = 0; e < q.ni; ++e) post[e] = YU[(int64_t)e * nc + j];
        for (int r = 0; r < q.nc; ++r) post[q.ni + r] = YP[(int64_t)r * nc + j];
        for (int k = 0; k < q.ng; ++k) {
            const int64_t gk = v.o_ng[q.s] + k;
            const int r = v.gcell[gk], a = v.gaxis[gk], side = v.gside[gk];
            const int64_t cb = (v.o_cell[q.s] + r) * 3;
            const double sc = v.cs[cb + a];
            const int other = side == 0 ? v.chi[cb + a] : v.clo[cb + a];
            double val = q.d * (side == 0 ? 1.0 : -1.0) * YP[(int64_t)r * nc + j];
            if (other >= q.ng) val += kMassOffD * sc * YU[(int64_t)(other - q.ng) * nc + j];
            if (j < q.ng) {
                if (k == j) val += kMassDiagD * sc;
                if (other >= 0 && other < q.ng && other == j) val += kMassOffD * sc;
                v.S[v.o_S[q.s] + (int64_t)j * q.ng + k] = val;
            } else {
                v.GpreT[v.o_Gpre[q.s] + (int64_t)(j - q.ng) * q.ng + k] = val;
            }
        }
    }
}

}  // namespace

namespace {

// device buffers of one call, freed together
struct DevBufs {
    std::vector<void*> ptrs;
    bool ok = true;
    template <class T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (!ok || cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    template <class T>
    T* upload(const std::vector<T>& v, cudaStream_t st) {
        T* p = alloc<T>(v.size());
        if (p && !v.empty() && cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
            ok = false;
        return p;
    }
    ~DevBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
};

constexpr size_t kScratchLimit = size_t(3) << 30;  // scratch of one launch chunk
constexpr int kChunkSubs = 8192;

}  // namespace

int local_maps_device(LocalMapsBatch& B, std::string& err) {
    const int n = B.n_sub;
    B.S.assign((size_t)B.o_S[n], 0.0);
    B.GpreT.assign((size_t)B.o_Gpre[n], 0.0);
    B.dev_GpostT.reset();
    B.status.assign(n, BDDC_OK);
    if (n == 0) return BDDC_OK;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        err = "stream";
        return BDDC_E_CUDA;
    }
    int rc = BDDC_OK;
    {
        DevBufs m;
        LmView v{};
        v.dim = m.upload(B.dim, st);
        v.ng = m.upload(B.ng, st);
        v.ni = m.upload(B.ni, st);
        v.nc = m.upload(B.nc, st);
        v.vol = m.upload(B.vol, st);
        v.d = m.upload(B.d, st);
        v.o_cell = m.upload(B.o_cell, st);
        v.o_ng = m.upload(B.o_ng, st);
        v.o_ni = m.upload(B.o_ni, st);
        v.o_ch = m.upload(B.o_ch, st);
        v.o_S = m.upload(B.o_S, st);
        v.o_Gpre = m.upload(B.o_Gpre, st);
        v.o_Gpost = m.upload(B.o_Gpost, st);
        v.clo = m.upload(B.clo, st);
        v.chi = m.upload(B.chi, st);
        v.cs = m.upload(B.cs, st);
        v.gcell = m.upload(B.gcell, st);
        v.gaxis = m.upload(B.gaxis, st);
        v.gside = m.upload(B.gside, st);
        v.order = m.upload(B.order, st);
        v.cstart = m.upload(B.cstart, st);
        v.rdfac = m.upload(B.rdfac, st);
        v.lfac = m.upload(B.lfac, st);
        v.off = m.upload(B.off, st);
        v.S = m.alloc<double>(B.S.size());
        v.GpreT = m.alloc<double>(B.GpreT.size());
        {
            // G_post stays on the device for the solve handle: owned by a shared pointer
            void* gp = nullptr;
            if (cudaMalloc(&gp, std::max<int64_t>(B.o_Gpost[n], 1) * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                m.ok = false;
            } else {
                B.dev_GpostT = std::shared_ptr<double>(static_cast<double*>(gp), [](double* q) { cudaFree(q); });
            }
            v.GpostT = B.dev_GpostT.get();
        }
        v.status = m.upload(B.status, st);
        // chunks of subdomains whose scratch fits the limit
        std::vector<int> cuts{0};
        std::vector<std::vector<int64_t>> offs;  // per chunk: Y, Q, U, P, piv offsets
        size_t max_Y = 0, max_Q = 0, max_U = 0, max_P = 0, max_piv = 0;
        {
            std::vector<int64_t> oY{0}, oQ{0}, oU{0}, oP{0}, oV{0};
            auto close = [&](int end) {
                max_Y = std::max<size_t>(max_Y, oY.back());
                max_Q = std::max<size_t>(max_Q, oQ.back());
                max_U = std::max<size_t>(max_U, oU.back());
                max_P = std::max<size_t>(max_P, oP.back());
                max_piv = std::max<size_t>(max_piv, oV.back());
                std::vector<int64_t> all;
                for (auto* o : {&oY, &oQ, &oU, &oP, &oV}) all.insert(all.end(), o->begin(), o->end());
                offs.push_back(all);
                cuts.push_back(end);
                for (auto* o : {&oY, &oQ, &oU, &oP, &oV}) o->assign(1, 0);
            };
            for (int s = 0; s < n; ++s) {
                const int64_t ni = B.ni[s], nc = B.nc[s], nq = nc + 1, ncol = B.ng[s] + nc;
                const size_t add = 8 * (size_t)(ni * nc + nq * nq + 4 * ni * ncol + 4 * nq * ncol) + 4 * nq;
                const size_t cur = 8 * (size_t)(oY.back() + oQ.back() + 4 * oU.back() + 4 * oP.back()) + 4 * oV.back();
                if (s > cuts.back() && (cur + add > kScratchLimit || s - cuts.back() >= kChunkSubs)) close(s);
                oY.push_back(oY.back() + ni * nc);
                oQ.push_back(oQ.back() + nq * nq);
                oU.push_back(oU.back() + ni * ncol);
                oP.push_back(oP.back() + nq * ncol);
                oV.push_back(oV.back() + nq);
            }
            close(n);
        }
        v.Y = m.alloc<double>(max_Y);
        v.Q = m.alloc<double>(max_Q);
        v.XU = m.alloc<double>(max_U);
        v.YU = m.alloc<double>(max_U);
        v.RU = m.alloc<double>(max_U);
        v.DU = m.alloc<double>(max_U);
        v.XP = m.alloc<double>(max_P);
        v.YP = m.alloc<double>(max_P);
        v.RP = m.alloc<double>(max_P);
        v.DP = m.alloc<double>(max_P);
        v.piv = m.alloc<int>(max_piv);
        int max_nq = 1;
        for (int s = 0; s < n; ++s) max_nq = std::max(max_nq, B.nc[s] + 1);
        if (!m.ok) {
            rc = BDDC_E_OOM;
            err = "device memory for the local maps";
        }
        for (size_t c = 0; rc == BDDC_OK && c + 1 < cuts.size(); ++c) {
            const int s0 = cuts[c], cnt = cuts[c + 1] - cuts[c];
            DevBufs mc;
            const std::vector<int64_t>& all = offs[c];
            const size_t k = (size_t)cnt + 1;
            int64_t* o = mc.upload(all, st);
            if (!mc.ok) {
                rc = BDDC_E_OOM;
                err = "device memory for the local maps";
                break;
            }
            v.sub0 = s0;
            v.o_Y = o;
            v.o_Q = o + k;
            v.o_U = o + 2 * k;
            v.o_P = o + 3 * k;
            v.o_piv = o + 4 * k;
            k_lm_Y<<<cnt, kLmThreads, 0, st>>>(v);
            k_lm_Q<<<cnt, kLmThreads, 0, st>>>(v);
            k_lm_lu<<<cnt, kLmThreads, sizeof(double) * max_nq, st>>>(v);
            k_lm_rhs<<<cnt, kLmThreads, 0, st>>>(v);
            k_lm_solve<<<cnt, kLmThreads, 0, st>>>(v, v.XU, v.XP, v.YU, v.YP);
            const int64_t nU = all[2 * k + cnt], nP = all[3 * k + cnt];
            for (int pass = 0; pass < kLocalRefinements; ++pass) {
                k_lm_resid<<<cnt, kLmThreads, 0, st>>>(v);
                k_lm_solve<<<cnt, kLmThreads, 0, st>>>(v, v.RU, v.RP, v.DU, v.DP);
                k_lm_add<<<(int)std::min<int64_t>((nU + 255) / 256, 65536), 256, 0, st>>>(nU, v.YU, v.DU);
                k_lm_add<<<(int)std::min<int64_t>((nP + 255) / 256, 65536), 256, 0, st>>>(nP, v.YP, v.DP);
            }
            k_lm_out<<<cnt, kLmThreads, 0, st>>>(v);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                rc = BDDC_E_CUDA;
                err = cudaGetErrorString(cudaGetLastError());
            }
        }
        if (rc == BDDC_OK) {
            cudaMemcpyAsync(B.S.data(), v.S, B.S.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(B.GpreT.data(), v.GpreT, B.GpreT.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(B.status.data(), v.status, B.status.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                rc = BDDC_E_CUDA;
                err = cudaGetErrorString(cudaGetLastError());
            }
        }
    }
    cudaStreamDestroy(st);
    if (rc != BDDC_OK) B.dev_GpostT.reset();
    return rc;
}

bool device_to_host(const double* dev, int64_t n, double* host) {
    return n <= 0 || cudaMemcpy(host, dev, n * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
}

}  // namespace bddc

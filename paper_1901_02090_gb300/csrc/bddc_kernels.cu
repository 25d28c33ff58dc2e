// GB300 (sm_103a) kernels and C ABI of the BDDC solver.
//
// The solve is one persistent cooperative kernel (bddc_solve_kernel) per
// batch of instances.  Its phases follow Algorithm 1 of the paper:
//   Step 1  coarse right-hand side, coarse solve, u_0 = E w_0;
//   Step 2  local residuals S u_0 + G f of the subdomain problems, giving the
//           reduced right-hand side f* of eqs. (corr-reduced-1/2);
//   Step 3  CG on the pairs (w_hat, p_0) with the BDDC preconditioner of
//           Algorithm 2; per iteration four phases:
//             DIROP   d = z + beta d, q = S d + B_0^T d_p       (rows a1, a2)
//             UPDATE  x += alpha d, r -= alpha q, restrict r,
//                     subdomain correction F r, Psi^T r          (a2, a3, a4, a6)
//             COARSE  coarse solve                               (a5)
//             PROLONG z = E (Psi w_c + F r), (r, z)             (a7, a8)
//   post    interiors and pressures from the final interface flux.
// The iterations, the inner products and the coarse solve are FP64; the
// subdomain-correction operator F and the coarse basis Psi are FP64 or FP32.
//
// Every reduction is a fixed-order sum of per-subdomain partials, so all CTAs
// reach bit-identical scalars and take the same decisions.  Every interface
// value that two subdomains share is recomputed by both (a + b is
// commutative in IEEE arithmetic) and stored once, by its owner slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bddc_internal.hpp"
#include "bddc_kernels.cuh"
#include "dense.hpp"

namespace bddc {

// ---- small device helpers --------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order block sum; `red` holds >= 16 doubles of shared memory
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) r += red[i];
        red[8] = r;
    }
    __syncthreads();
    const double r = red[8];
    __syncthreads();
    return r;
}

// fixed-order sum of part[s0..s1) by warp 0, broadcast to the block
__device__ double range_sum(const double* part, int64_t s0, int64_t s1, double* red) {
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int64_t s = s0 + threadIdx.x; s < s1; s += 32) v += __ldcg(part + s);
        v = warp_sum(v);
        if (threadIdx.x == 0) red[9] = v;
    }
    __syncthreads();
    const double r = red[9];
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool slot_owner(int slot, int partner) { return partner < 0 || slot < partner; }

__device__ __forceinline__ int inst_done(const Params& p, int b) {
    return __ldcg(&p.st[b].done);
}

// grid-wide barrier with a bounded wait; false if any CTA gave up
__device__ bool grid_barrier(GridSync* gs) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &gs->gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&gs->count, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == g0) {
                if (++spins > kSpinLimit) { ok = 0; break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (!ok) atomicExch(&gs->error, 1);
        if (*(volatile int*)&gs->error) ok = 0;
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

__device__ __forceinline__ void my_range(int64_t U, int64_t& a, int64_t& b) {
    a = (U * (int64_t)blockIdx.x) / gridDim.x;
    b = (U * ((int64_t)blockIdx.x + 1)) / gridDim.x;
}

template <class T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };

// Shared-memory layout of one CTA (dynamic): xs[max_ng] doubles,
// xin[max_in_post] doubles, rhs[max_ncn] doubles, xsf[max_ng] floats,
// red[16] doubles.
struct Smem {
    double *xs, *xin, *rhs, *red;
    float* xsf;
};
__device__ __forceinline__ Smem carve(const Params& p, double* base) {
    Smem s;
    s.xs = base;
    s.xin = s.xs + p.max_ng;
    s.rhs = s.xin + p.max_in_post;
    s.red = s.rhs + p.max_ncn;
    s.xsf = reinterpret_cast<float*>(s.red + 16);
    return s;
}

// y_i = (sum_j M[j*n + i] * v_j), thread per output, inputs in shared memory
template <class T, class A>
__device__ __forceinline__ A gemv_col(const T* __restrict__ M, int n_out, int n_in, const A* v, int o) {
    A acc = 0;
#pragma unroll 4
    for (int j = 0; j < n_in; ++j) acc += (A)__ldg(M + (int64_t)j * n_out + o) * v[j];
    return acc;
}

// subdomain correction and coarse restriction of the weighted residual in
// sm.xs: yl = F xs, rcl = Psi^T xs (Algorithm 2 steps 1-2, local parts)
template <class T>
__device__ void restrict_apply(const Params& p, int64_t s, Smem& sm) {
    using A = typename Acc<T>::type;
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const T* F = reinterpret_cast<const T*>(p.F) + p.off_F[s];
    const T* P = reinterpret_cast<const T*>(p.P) + p.off_P[s];
    const A* v;
    if constexpr (sizeof(T) == 4) {
        for (int k = threadIdx.x; k < ng; k += kThreads) sm.xsf[k] = (float)sm.xs[k];
        __syncthreads();
        v = reinterpret_cast<const A*>(sm.xsf);
    } else {
        v = reinterpret_cast<const A*>(sm.xs);
    }
    for (int k = threadIdx.x; k < ng; k += kThreads) p.yl[so + k] = (double)gemv_col<T, A>(F, ng, ng, v, k);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int a = w; a < m; a += kThreads / 32) {
        A acc = 0;
        for (int k = l; k < ng; k += 32) acc += (A)__ldg(P + (int64_t)a * ng + k) * v[k];
        double d = (double)acc;
        d = warp_sum(d);
        if (l == 0) p.rcl[co + a] = d;
    }
    __syncthreads();
}

// z_loc = Psi * wc_local (+ add), thread per output; wc staged in sm.rhs
template <class T>
__device__ __forceinline__ double prolong_one(const Params& p, int64_t s, int ng, int m, const double* wcs, int k) {
    const T* P = reinterpret_cast<const T*>(p.P) + p.off_P[s];
    using A = typename Acc<T>::type;
    A acc = 0;
    for (int a = 0; a < m; ++a) acc += (A)__ldg(P + (int64_t)a * ng + k) * (A)wcs[a];
    return (double)acc;
}

__device__ void stage_wc(const Params& p, int64_t s, const double* wc_b, Smem& sm) {
    const int m = p.sub_m[s];
    const int64_t co = p.off_cslot[s];
    for (int a = threadIdx.x; a < m; a += kThreads) sm.rhs[a] = __ldcg(wc_b + p.cslot_c[co + a]);
    __syncthreads();
}

// ---- phases -------------------------------------------------------------------------
template <class T>
__device__ void ph_step1(const Params& p, int64_t s, Smem& sm) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    for (int k = threadIdx.x; k < ng; k += kThreads) {
        const int gi = p.slot_g[so + k];
        const double sg = p.g_bsign[gi];
        const double gv = sg != 0.0 ? sg * p.bc_in[p.g_fid[gi]] : 0.0;
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.g[gi] = gv;
        sm.xs[k] = p.slot_w[so + k] * gv;
    }
    __syncthreads();
    using A = typename Acc<T>::type;
    const T* P = reinterpret_cast<const T*>(p.P) + p.off_P[s];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int a = w; a < m; a += kThreads / 32) {
        double acc = 0.0;  // Step 1 right-hand side in FP64 products
        for (int k = l; k < ng; k += 32) acc += (double)(A)__ldg(P + (int64_t)a * ng + k) * sm.xs[k];
        acc = warp_sum(acc);
        if (l == 0) p.rcl[co + a] = acc;
    }
    double v = 0.0;
    const int64_t cb = p.off_cell[s];
    for (int r = threadIdx.x; r < nc; r += kThreads) v += -p.f_in[p.cell_gid[cb + r]];
    v = block_sum(v, sm.red);
    if (threadIdx.x == 0) p.prhs[s] = p.sub_d[s] * p.inst_vol[b] * v;
    __syncthreads();
}

// coarse solve rows: wc = Kinv * rhs (rhs flux part from coarse slots; the
// pressure part is the Step-1 right-hand side or zero)
__device__ void ph_coarse(const Params& p, int64_t u, bool step1, Smem& sm, int& staged) {
    const int b = p.cunit_inst[u];
    if (!step1 && inst_done(p, b)) return;
    const int64_t ncn = p.inst_ncn[b], ncf = p.inst_ncf[b], coff = p.inst_coff[b];
    const int64_t cfo = p.inst_cfoff[b];
    const int64_t ncols = step1 ? ncn : ncf;
    if (staged != b) {
        __syncthreads();
        const int64_t s0 = p.inst_s0[b];
        for (int64_t c = threadIdx.x; c < ncols; c += kThreads) {
            double v;
            if (c < ncf) {
                const int a = p.c_slot_a[cfo + c], bb = p.c_slot_b[cfo + c];
                v = (a >= 0 ? __ldcg(p.rcl + a) : 0.0) + (bb >= 0 ? __ldcg(p.rcl + bb) : 0.0);
            } else {
                v = __ldcg(p.prhs + s0 + (c - ncf));
            }
            sm.rhs[c] = v;
        }
        __syncthreads();
        staged = b;
    }
    const double* K = p.Kinv + p.inst_kinv_off[b];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t r0 = p.cunit_row0[u];
    const int64_t r1 = (r0 + kCoarseRows < ncn) ? r0 + kCoarseRows : ncn;
    for (int64_t row = r0 + w; row < r1; row += kThreads / 32) {
        const double* kr = K + row * ncn;
        double acc = 0.0;
        for (int64_t c = l; c < ncols; c += 32) acc += __ldg(kr + c) * sm.rhs[c];
        acc = warp_sum(acc);
        if (l == 0) p.wc[coff + row] = acc;
    }
}

template <class T>
__device__ void ph_u0(const Params& p, int64_t s, Smem& sm) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s];
    stage_wc(p, s, p.wc + p.inst_coff[b], sm);
    for (int k = threadIdx.x; k < ng; k += kThreads)
        p.tl[so + k] = p.slot_w[so + k] * prolong_one<T>(p, s, ng, m, sm.rhs, k);
    __syncthreads();
}

// Step 2 local residual r_G = S u_0 + G_pre f (stored in ql)
__device__ void ph_step2(const Params& p, int64_t s, Smem& sm) {
    const int ng = p.sub_ng[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], cb = p.off_cell[s];
    for (int k = threadIdx.x; k < ng; k += kThreads) {
        const int pt = p.slot_partner[so + k];
        const double u = __ldcg(p.tl + so + k) + (pt >= 0 ? __ldcg(p.tl + pt) : 0.0);
        if (slot_owner((int)(so + k), pt)) p.u0[p.slot_g[so + k]] = u;
        sm.xin[k] = u;
    }
    for (int r = threadIdx.x; r < nc; r += kThreads) sm.xin[ng + r] = p.f_in[p.cell_gid[cb + r]];
    __syncthreads();
    const double* S = p.S + p.off_S[s];
    const double* G = p.Gpre + p.off_Gpre[s];
    for (int k = threadIdx.x; k < ng; k += kThreads)
        p.ql[so + k] = gemv_col<double, double>(S, ng, ng, sm.xin, k) +
                       gemv_col<double, double>(G, ng, nc, sm.xin + ng, k);
    __syncthreads();
}

// f* = g - sum_i R_i^T r_G,i ; r_0 = f*, x_0 = 0 ; then restrict r_0
template <class T>
__device__ void ph_fstar(const Params& p, int64_t s, Smem& sm) {
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    double rr = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = threadIdx.x; k < ng; k += kThreads) {
        const int pt = p.slot_partner[so + k];
        const int gi = p.slot_g[so + k];
        const double gv = __ldcg(p.g + gi);
        const double loc = __ldcg(p.ql + so + k) + (pt >= 0 ? __ldcg(p.ql + pt) : 0.0);
        const double fs = gv - loc;
        if (slot_owner((int)(so + k), pt)) {
            p.rbuf0[gi] = fs;
            p.x[gi] = 0.0;
            rr += fs * fs;
            a1 += gv * gv;
            a2 += loc * loc;
        }
        const double wr = p.slot_w[so + k] * fs;
        sm.xs[k] = wr;
        p.rl[so + k] = wr;
    }
    rr = block_sum(rr, sm.red);
    a1 = block_sum(a1, sm.red);
    a2 = block_sum(a2, sm.red);
    if (threadIdx.x == 0) {
        p.part_rr[s] = rr;
        p.part_a1[s] = a1;
        p.part_a2[s] = a2;
        p.xp[s] = 0.0;
        p.dp0[s] = 0.0;
        p.dp1[s] = 0.0;
    }
    __syncthreads();
    restrict_apply<T>(p, s, sm);
}

template <class T>
__device__ void ph_prolong(const Params& p, int64_t s, Smem& sm) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return;
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s];
    const double* wcb = p.wc + p.inst_coff[b];
    stage_wc(p, s, wcb, sm);
    double rz = 0.0;
    for (int k = threadIdx.x; k < ng; k += kThreads) {
        const double z = prolong_one<T>(p, s, ng, m, sm.rhs, k) + __ldcg(p.yl + so + k);
        p.zl[so + k] = p.slot_w[so + k] * z;
        rz += __ldcg(p.rl + so + k) * z;
    }
    rz = block_sum(rz, sm.red);
    if (threadIdx.x == 0) {
        p.part_rz[s] = rz;
        p.zp[s] = __ldcg(wcb + p.inst_ncf[b] + p.sub_local[s]);
    }
    __syncthreads();
}

constexpr double kRhoFluxConverged = 1e-24;

// convergence decision, direction update and operator apply
__device__ void ph_dirop(const Params& p, int64_t s, int k, Smem& sm) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return;
    const int64_t s0 = p.inst_s0[b], s1 = p.inst_s1[b];
    const double rr = range_sum(p.part_rr, s0, s1, sm.red);
    const double rz = range_sum(p.part_rz, s0, s1, sm.red);
    const bool owner = (s == s0);
    const int64_t hb = (int64_t)b * (p.maxit + 1);
    double r0, floor_, rho0;
    if (k == 0) {
        const double a1 = range_sum(p.part_a1, s0, s1, sm.red);
        const double a2 = range_sum(p.part_a2, s0, s1, sm.red);
        r0 = sqrt(rr);
        floor_ = 1e-14 * (sqrt(a1) + sqrt(a2));
        rho0 = rz;
    } else {
        r0 = __ldcg(&p.st[b].r0);
        floor_ = __ldcg(&p.st[b].floor);
        rho0 = __ldcg(&p.st[b].rho0);
    }
    const double nr = sqrt(rr);
    const double relres = (k == 0) ? 1.0 : nr / r0;
    int status = -100;  // not done
    if (k == 0) {
        if (nr <= floor_) status = BDDC_OK;
        else if (!(rz > 0.0)) status = BDDC_E_BREAKDOWN;
    } else {
        if (relres <= p.tol || nr <= floor_ || rz <= kRhoFluxConverged * rho0) status = BDDC_OK;
        else if (!(rz > 0.0)) status = BDDC_E_BREAKDOWN;
        else if (k >= p.maxit) status = BDDC_E_NOT_CONVERGED;
    }
    if (owner) {
        if (threadIdx.x == 0) {
            if (k == 0) {
                p.st[b].r0 = r0;
                p.st[b].floor = floor_;
                p.st[b].rho0 = rho0;
            }
            p.rho_hist[hb + k] = rz;
        }
        if (status != -100) {
            // last coarse pressure correction x_p += z_p from the final residual
            for (int64_t t = s0 + threadIdx.x; t < s1; t += kThreads) p.xp[t] = __ldcg(p.xp + t) + __ldcg(p.zp + t);
            if (threadIdx.x == 0) {
                p.st[b].status = status;
                p.st[b].iterations = k;
                p.st[b].relres = relres;
                __threadfence();
                p.st[b].done = 1;
                atomicSub(p.n_active, 1);
            }
        }
    }
    if (status != -100) return;
    const double beta = (k == 0) ? 0.0 : rz / __ldcg(p.rho_hist + hb + k - 1);
    if (owner && threadIdx.x == 0) p.beta_hist[hb + k] = beta;
    double* dold = (k & 1) ? p.dbuf0 : p.dbuf1;
    double* dnew = (k & 1) ? p.dbuf1 : p.dbuf0;
    double* dpold = (k & 1) ? p.dp0 : p.dp1;
    double* dpnew = (k & 1) ? p.dp1 : p.dp0;
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    for (int kk = threadIdx.x; kk < ng; kk += kThreads) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        const double z = __ldcg(p.zl + so + kk) + (pt >= 0 ? __ldcg(p.zl + pt) : 0.0);
        const double dn = (k == 0) ? z : z + beta * __ldcg(dold + gi);
        if (slot_owner((int)(so + kk), pt)) dnew[gi] = dn;
        sm.xs[kk] = dn;
    }
    const double dpn = (k == 0) ? __ldcg(p.zp + s) : __ldcg(p.zp + s) + beta * __ldcg(dpold + s);
    if (threadIdx.x == 0) dpnew[s] = dpn;
    __syncthreads();
    const double* S = p.S + p.off_S[s];
    double dq = 0.0;
    for (int kk = threadIdx.x; kk < ng; kk += kThreads) {
        const double q = gemv_col<double, double>(S, ng, ng, sm.xs, kk) + p.slot_dsig[so + kk] * dpn;
        p.ql[so + kk] = q;
        dq += sm.xs[kk] * q;
    }
    dq = block_sum(dq, sm.red);
    if (threadIdx.x == 0) p.part_dq[s] = dq;
    __syncthreads();
}

template <class T>
__device__ void ph_update(const Params& p, int64_t s, int k, Smem& sm) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return;
    const int64_t s0 = p.inst_s0[b], s1 = p.inst_s1[b];
    const int64_t hb = (int64_t)b * (p.maxit + 1);
    const double dq = range_sum(p.part_dq, s0, s1, sm.red);
    const bool owner = (s == s0);
    if (!(dq > 0.0)) {
        if (owner && threadIdx.x == 0) {
            p.st[b].status = BDDC_E_BREAKDOWN;
            p.st[b].iterations = k;
            p.st[b].relres = -1.0;
            __threadfence();
            p.st[b].done = 1;
            atomicSub(p.n_active, 1);
        }
        return;
    }
    const double alpha = __ldcg(p.rho_hist + hb + k) / dq;
    if (owner && threadIdx.x == 0) p.alpha_hist[hb + k] = alpha;
    const double* rold = (k & 1) ? p.rbuf1 : p.rbuf0;
    double* rnew = (k & 1) ? p.rbuf0 : p.rbuf1;
    const double* dcur = (k & 1) ? p.dbuf1 : p.dbuf0;
    const double* dpcur = (k & 1) ? p.dp1 : p.dp0;
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    double rr = 0.0;
    for (int kk = threadIdx.x; kk < ng; kk += kThreads) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        const double q = __ldcg(p.ql + so + kk) + (pt >= 0 ? __ldcg(p.ql + pt) : 0.0);
        const double rn = __ldcg(rold + gi) - alpha * q;
        if (slot_owner((int)(so + kk), pt)) {
            rnew[gi] = rn;
            p.x[gi] = __ldcg(p.x + gi) + alpha * __ldcg(dcur + gi);
            rr += rn * rn;
        }
        const double wr = p.slot_w[so + kk] * rn;
        sm.xs[kk] = wr;
        p.rl[so + kk] = wr;
    }
    rr = block_sum(rr, sm.red);
    if (threadIdx.x == 0) {
        p.part_rr[s] = rr;
        p.xp[s] = __ldcg(p.xp + s) + alpha * __ldcg(dpcur + s);
    }
    __syncthreads();
    restrict_apply<T>(p, s, sm);
}

__device__ void ph_post(const Params& p, int64_t s, Smem& sm) {
    const int ng = p.sub_ng[s], ni = p.sub_ni[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], cb = p.off_cell[s], ib = p.off_int[s];
    for (int k = threadIdx.x; k < ng; k += kThreads) {
        const int gi = p.slot_g[so + k];
        const double u = __ldcg(p.u0 + gi) + __ldcg(p.x + gi);
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.flux_out[p.g_fid[gi]] = u;
        sm.xin[k] = u;
    }
    for (int r = threadIdx.x; r < nc; r += kThreads) sm.xin[ng + r] = p.f_in[p.cell_gid[cb + r]];
    __syncthreads();
    const double* G = p.Gpost + p.off_Gpost[s];
    const int no = ni + nc;
    const double d = p.sub_d[s];
    const double xp = __ldcg(p.xp + s);
    for (int o = threadIdx.x; o < no; o += kThreads) {
        const double v = gemv_col<double, double>(G, no, ng + nc, sm.xin, o);
        if (o < ni) p.flux_out[p.int_fid[ib + o]] = v;
        else p.p_out[p.cell_gid[cb + o - ni]] = d * (xp + v);
    }
    __syncthreads();
}

// ---- the persistent solve kernel -------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) bddc_solve_kernel(Params p) {
    extern __shared__ double smem_base[];
    Smem sm = carve(p, smem_base);
    int64_t a, e;
    int staged;
    my_range(p.n_sub, a, e);
    for (int64_t s = a; s < e; ++s) ph_step1<T>(p, s, sm);
    if (!grid_barrier(p.gsync)) return;
    staged = -1;
    my_range(p.n_cunits, a, e);
    for (int64_t u = a; u < e; ++u) ph_coarse(p, u, true, sm, staged);
    if (!grid_barrier(p.gsync)) return;
    my_range(p.n_sub, a, e);
    for (int64_t s = a; s < e; ++s) ph_u0<T>(p, s, sm);
    if (!grid_barrier(p.gsync)) return;
    for (int64_t s = a; s < e; ++s) ph_step2(p, s, sm);
    if (!grid_barrier(p.gsync)) return;
    for (int64_t s = a; s < e; ++s) ph_fstar<T>(p, s, sm);
    if (!grid_barrier(p.gsync)) return;
    staged = -1;
    my_range(p.n_cunits, a, e);
    for (int64_t u = a; u < e; ++u) ph_coarse(p, u, false, sm, staged);
    if (!grid_barrier(p.gsync)) return;
    my_range(p.n_sub, a, e);
    for (int64_t s = a; s < e; ++s) ph_prolong<T>(p, s, sm);
    if (!grid_barrier(p.gsync)) return;
    for (int k = 0;; ++k) {
        my_range(p.n_sub, a, e);
        for (int64_t s = a; s < e; ++s) ph_dirop(p, s, k, sm);
        if (!grid_barrier(p.gsync)) return;
        if (__ldcg(p.n_active) <= 0) break;
        for (int64_t s = a; s < e; ++s) ph_update<T>(p, s, k, sm);
        if (!grid_barrier(p.gsync)) return;
        staged = -1;
        my_range(p.n_cunits, a, e);
        for (int64_t u = a; u < e; ++u) ph_coarse(p, u, false, sm, staged);
        if (!grid_barrier(p.gsync)) return;
        my_range(p.n_sub, a, e);
        for (int64_t s = a; s < e; ++s) ph_prolong<T>(p, s, sm);
        if (!grid_barrier(p.gsync)) return;
    }
    my_range(p.n_sub, a, e);
    for (int64_t s = a; s < e; ++s) ph_post(p, s, sm);
}

// ---- stand-alone operator / preconditioner kernels (grid-stride over units) --------
__global__ void __launch_bounds__(kThreads) k_operator_local(Params p, const double* u, const double* p0) {
    extern __shared__ double smem_base[];
    Smem sm = carve(p, smem_base);
    for (int64_t s = blockIdx.x; s < p.n_sub; s += gridDim.x) {
        const int ng = p.sub_ng[s];
        const int64_t so = p.off_slot[s];
        for (int k = threadIdx.x; k < ng; k += kThreads) sm.xs[k] = u[p.slot_g[so + k]];
        __syncthreads();
        const double* S = p.S + p.off_S[s];
        const double pv = p0[s];
        for (int k = threadIdx.x; k < ng; k += kThreads)
            p.ql[so + k] = gemv_col<double, double>(S, ng, ng, sm.xs, k) + p.slot_dsig[so + k] * pv;
        __syncthreads();
    }
}

__global__ void k_assemble(int64_t n_slots, const double* loc, const int* slot_g, const int* partner, double* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_slots; q += (int64_t)gridDim.x * blockDim.x) {
        const int pt = partner[q];
        if (pt >= 0 && pt < q) continue;
        out[slot_g[q]] = loc[q] + (pt >= 0 ? loc[pt] : 0.0);
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_precond_restrict(Params p, const double* r) {
    extern __shared__ double smem_base[];
    Smem sm = carve(p, smem_base);
    for (int64_t s = blockIdx.x; s < p.n_sub; s += gridDim.x) {
        const int ng = p.sub_ng[s];
        const int64_t so = p.off_slot[s];
        for (int k = threadIdx.x; k < ng; k += kThreads) {
            const double wr = p.slot_w[so + k] * r[p.slot_g[so + k]];
            sm.xs[k] = wr;
            p.rl[so + k] = wr;
        }
        __syncthreads();
        restrict_apply<T>(p, s, sm);
    }
}

__global__ void __launch_bounds__(kThreads) k_precond_coarse(Params p) {
    extern __shared__ double smem_base[];
    Smem sm = carve(p, smem_base);
    int staged = -1;
    for (int64_t u = blockIdx.x; u < p.n_cunits; u += gridDim.x) {
        staged = -1;
        ph_coarse(p, u, false, sm, staged);
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_precond_prolong(Params p, double* z0) {
    extern __shared__ double smem_base[];
    Smem sm = carve(p, smem_base);
    for (int64_t s = blockIdx.x; s < p.n_sub; s += gridDim.x) {
        const int b = p.sub_inst[s];
        const int ng = p.sub_ng[s], m = p.sub_m[s];
        const int64_t so = p.off_slot[s];
        const double* wcb = p.wc + p.inst_coff[b];
        stage_wc(p, s, wcb, sm);
        for (int k = threadIdx.x; k < ng; k += kThreads)
            p.zl[so + k] = p.slot_w[so + k] * (prolong_one<T>(p, s, ng, m, sm.rhs, k) + p.yl[so + k]);
        if (threadIdx.x == 0) z0[s] = wcb[p.inst_ncf[b] + p.sub_local[s]];
        __syncthreads();
    }
}

// raw subassembled apply (no handle)
__global__ void __launch_bounds__(kThreads) k_subassembled_local(int n_sub, const int* ng_arr, const int64_t* slot_off,
                                                                 const int64_t* S_off, const double* S, const int* gidx,
                                                                 const double* u, double* scratch) {
    __shared__ double xs[1024];
    for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
        const int ng = ng_arr[s];
        const int64_t so = slot_off[s];
        for (int k = threadIdx.x; k < ng; k += blockDim.x) xs[k] = u[gidx[so + k]];
        __syncthreads();
        const double* M = S + S_off[s];
        for (int k = threadIdx.x; k < ng; k += blockDim.x) scratch[so + k] = gemv_col<double, double>(M, ng, ng, xs, k);
        __syncthreads();
    }
}

}  // namespace bddc

// ===================================================================================
// C ABI
// ===================================================================================
using namespace bddc;

struct bddc_handle {
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_inst = 0, maxit = 0, precision = 0;
    Packed P;
    Params prm{};
    std::vector<void*> allocs;
    std::string err;
    std::vector<bddc_stats> stats;
    std::vector<int64_t> inst_cfoff;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float last_ms = 0.0f;
    double last_bytes = 0.0;
    int grid = 0;
    size_t smem = 0;
    int64_t total_cells = 0, total_faces = 0;
    double *d_f = nullptr, *d_bc = nullptr, *d_flux = nullptr, *d_p = nullptr;
    double* d_hist_a = nullptr;
    int64_t* d_cfoff = nullptr;
    double bytes_iter = 0.0, bytes_pre = 0.0, bytes_post = 0.0;
};

namespace {

const char* kErrStrings[] = {"ok", "invalid argument", "invalid partition", "invalid permeability",
                             "out of memory", "not converged", "CG breakdown", "device wait timed out",
                             "CUDA error", "setup factorisation failed"};

thread_local std::string g_setup_err;

int set_err(bddc_handle* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

template <class T>
int upload(bddc_handle* h, const std::vector<T>& v, const T** out) {
    *out = nullptr;
    if (v.empty()) return BDDC_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, v.size() * sizeof(T)) != cudaSuccess) return BDDC_E_OOM;
    h->allocs.push_back(p);
    if (cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return BDDC_E_CUDA;
    *out = static_cast<const T*>(p);
    return BDDC_OK;
}

template <class T>
int dalloc(bddc_handle* h, size_t n, T** out) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return BDDC_E_OOM;
    h->allocs.push_back(p);
    cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(T));
    *out = static_cast<T*>(p);
    return BDDC_OK;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void bddc_default_options(bddc_options* opt) {
    if (!opt) return;
    opt->tau = 0.0;
    opt->scaling = BDDC_SCALING_MULTIPLICITY;
    opt->precision = BDDC_PREC_FP64;
    opt->maxit = 5000;
    opt->pressure_scaling = 1;
    opt->n_threads = 0;
}

const char* bddc_error_string(int code) {
    const int i = -code;
    if (i < 0 || i >= (int)(sizeof(kErrStrings) / sizeof(kErrStrings[0]))) return "unknown error";
    return kErrStrings[i];
}

const char* bddc_last_error(const bddc_handle* h) { return h ? h->err.c_str() : g_setup_err.c_str(); }

void bddc_destroy(bddc_handle* h) {
    if (!h) return;
    for (void* p : h->allocs) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

int bddc_setup(int n_instances, const bddc_instance* inst, const bddc_options* opt_in, void* cuda_stream,
               bddc_handle** out) {
    g_setup_err.clear();
    if (!out) return BDDC_E_INVALID_ARG;
    *out = nullptr;
    if (n_instances <= 0 || !inst) return BDDC_E_INVALID_ARG;
    bddc_options opt;
    bddc_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.maxit <= 0 || (opt.precision != BDDC_PREC_FP64 && opt.precision != BDDC_PREC_FP32) ||
        (opt.scaling != BDDC_SCALING_MULTIPLICITY && opt.scaling != BDDC_SCALING_STIFFNESS))
        return BDDC_E_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return BDDC_E_CUDA;
    }
    bddc_handle* h = new bddc_handle();
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&h->device);
    h->n_inst = n_instances;
    h->maxit = opt.maxit;
    h->precision = opt.precision;
    SetupResult r = build_all(n_instances, inst, opt, h->P);
    if (r.code) {
        g_setup_err = r.msg;
        delete h;
        return r.code;
    }
    Packed& P = h->P;
    for (int b = 0; b < n_instances; ++b) {
        h->total_cells += P.inst_ncells[b];
        h->total_faces += P.inst_nfaces[b];
    }
    // coarse work units
    std::vector<int> cu_inst, cu_row0;
    for (int b = 0; b < n_instances; ++b)
        for (int64_t r0 = 0; r0 < P.inst_ncn[b]; r0 += kCoarseRows) {
            cu_inst.push_back(b);
            cu_row0.push_back((int)r0);
        }
    h->inst_cfoff.assign(n_instances, 0);
    for (int b = 1; b < n_instances; ++b) h->inst_cfoff[b] = h->inst_cfoff[b - 1] + P.inst_ncf[b - 1];
    Params& p = h->prm;
    int rc = BDDC_OK;
#define UP(field, vec) \
    if (!rc) rc = upload(h, vec, &p.field)
    UP(inst_goff, P.inst_goff); UP(inst_ng, P.inst_ng); UP(inst_coff, P.inst_coff); UP(inst_ncn, P.inst_ncn);
    UP(inst_ncf, P.inst_ncf); UP(inst_kinv_off, P.inst_kinv_off); UP(inst_s0, P.inst_s0); UP(inst_s1, P.inst_s1);
    UP(inst_vol, P.inst_vol);
    UP(sub_inst, P.sub_inst); UP(sub_ng, P.sub_ng); UP(sub_ni, P.sub_ni); UP(sub_nc, P.sub_nc);
    UP(sub_m, P.sub_m); UP(sub_local, P.sub_local);
    UP(off_S, P.off_S); UP(off_F, P.off_F); UP(off_P, P.off_P); UP(off_Gpre, P.off_Gpre); UP(off_Gpost, P.off_Gpost);
    UP(off_slot, P.off_slot); UP(off_cslot, P.off_cslot); UP(off_cell, P.off_cell); UP(off_int, P.off_int);
    UP(sub_d, P.sub_d); UP(slot_g, P.slot_g); UP(slot_partner, P.slot_partner); UP(slot_w, P.slot_w);
    UP(slot_dsig, P.slot_dsig); UP(cslot_c, P.cslot_c); UP(cell_gid, P.cell_gid); UP(int_fid, P.int_fid);
    UP(g_fid, P.g_fid); UP(g_bsign, P.g_bsign); UP(c_slot_a, P.c_slot_a); UP(c_slot_b, P.c_slot_b);
    UP(cunit_inst, cu_inst); UP(cunit_row0, cu_row0);
    UP(S, P.S); UP(Gpre, P.Gpre); UP(Gpost, P.Gpost); UP(Kinv, P.Kinv);
    UP(inst_cfoff, h->inst_cfoff);
#undef UP
    if (!rc) {
        if (opt.precision == BDDC_PREC_FP32) {
            const float *f = nullptr, *pp = nullptr;
            rc = upload(h, P.F32, &f);
            if (!rc) rc = upload(h, P.P32, &pp);
            p.F = f;
            p.P = pp;
        } else {
            const double *f = nullptr, *pp = nullptr;
            rc = upload(h, P.F64, &f);
            if (!rc) rc = upload(h, P.P64, &pp);
            p.F = f;
            p.P = pp;
        }
    }
    const int64_t G = P.n_gamma, L = P.off_slot.back(), CL = P.off_cslot.back(), NS = P.n_sub;
    const int64_t H = (int64_t)n_instances * (opt.maxit + 1);
#define AL(field, n) \
    if (!rc) rc = dalloc(h, (size_t)(n), &p.field)
    AL(x, G); AL(rbuf0, G); AL(rbuf1, G); AL(dbuf0, G); AL(dbuf1, G); AL(g, G); AL(u0, G);
    AL(ql, L); AL(zl, L); AL(yl, L); AL(rl, L); AL(tl, L);
    AL(rcl, CL); AL(wc, P.n_coarse_vec);
    AL(xp, NS); AL(dp0, NS); AL(dp1, NS); AL(zp, NS); AL(prhs, NS);
    AL(part_dq, NS); AL(part_rr, NS); AL(part_rz, NS); AL(part_a1, NS); AL(part_a2, NS);
    AL(st, n_instances); AL(alpha_hist, H); AL(beta_hist, H); AL(rho_hist, H);
    AL(n_active, 1); AL(gsync, 1);
#undef AL
    if (rc) {
        bddc_destroy(h);
        return rc;
    }
    p.n_inst = n_instances;
    p.n_sub = NS;
    p.n_cunits = (int64_t)cu_inst.size();
    p.maxit = opt.maxit;
    p.max_ng = std::max(P.max_ng, 1);
    p.max_in_post = std::max(P.max_in_post, 1);
    p.max_ncn = std::max(P.max_ncn, 1);
    h->smem = sizeof(double) * (size_t)(p.max_ng + p.max_in_post + p.max_ncn + 16) + sizeof(float) * (size_t)p.max_ng + 16;
    if (h->smem > 200 * 1024) {
        bddc_destroy(h);
        return BDDC_E_INVALID_ARG;  // coarse problem too large for the dense coarse solve
    }
    const void* kfn = opt.precision == BDDC_PREC_FP32 ? (const void*)bddc_solve_kernel<float>
                                                      : (const void*)bddc_solve_kernel<double>;
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem);
    int nb = 0, nsm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, kThreads, h->smem);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    const int64_t want = std::max<int64_t>(NS, p.n_cunits);
    h->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb * nsm, want));
    if (nb <= 0) {
        bddc_destroy(h);
        return BDDC_E_CUDA;
    }
    cudaEventCreate(&h->ev0);
    cudaEventCreate(&h->ev1);
    h->stats.assign(n_instances, bddc_stats{});
    for (int b = 0; b < n_instances; ++b) {
        h->stats[b].omega_tilde = P.inst_omega[b];
        h->stats[b].n_subdomains = (int)(P.inst_s1[b] - P.inst_s0[b]);
        h->stats[b].n_interface = (int)P.inst_ng[b];
        h->stats[b].n_coarse = (int)P.inst_ncn[b];
        h->stats[b].n_adaptive = P.inst_nadapt[b];
    }
    // algorithmic bytes (matrices once per use; vectors ~18 doubles per slot
    // and iteration)
    const double fb = opt.precision == BDDC_PREC_FP32 ? 4.0 : 8.0;
    double it_b = 0.0, pre_b = 0.0, post_b = 0.0;
    for (int64_t s = 0; s < NS; ++s) {
        const double ng = P.sub_ng[s], m = P.sub_m[s], nc = P.sub_nc[s], ni = P.sub_ni[s];
        it_b += 8.0 * ng * ng + fb * ng * ng + 2.0 * fb * m * ng + 8.0 * 18.0 * ng;
        pre_b += 3.0 * fb * m * ng + 8.0 * ng * ng + 8.0 * nc * ng + fb * ng * ng + 8.0 * 20.0 * ng;
        post_b += 8.0 * (ng + nc) * (ni + nc) + 8.0 * (ni + 2.0 * nc + 2.0 * ng);
    }
    for (int b = 0; b < n_instances; ++b) {
        const double ncn = P.inst_ncn[b], ncf = P.inst_ncf[b];
        it_b += 8.0 * ncn * ncf;
        pre_b += 8.0 * ncn * ncn + 8.0 * ncn * ncf;
    }
    h->bytes_iter = it_b;
    h->bytes_pre = pre_b;
    h->bytes_post = post_b;
    if (cudaGetLastError() != cudaSuccess) {
        bddc_destroy(h);
        return BDDC_E_CUDA;
    }
    *out = h;
    return BDDC_OK;
}

int bddc_sizes(const bddc_handle* h, int* n_instances, int64_t* n_interface, int64_t* n_subdomains) {
    if (!h) return BDDC_E_INVALID_ARG;
    if (n_instances) *n_instances = h->n_inst;
    if (n_interface) *n_interface = h->P.n_gamma;
    if (n_subdomains) *n_subdomains = h->P.n_sub;
    return BDDC_OK;
}

int bddc_solve(bddc_handle* h, const double* f, const double* bc_value, double tol, double* flux, double* pressure,
               int* iterations) {
    if (!h) return BDDC_E_INVALID_ARG;
    if (!f || !bc_value || !flux || !pressure || !(tol > 0.0) || !std::isfinite(tol))
        return set_err(h, BDDC_E_INVALID_ARG, "null array or non-positive tol");
    cudaSetDevice(h->device);
    cudaStream_t st = h->stream;
    const size_t ncell = (size_t)h->total_cells, nface = (size_t)h->total_faces;
    Params p = h->prm;
    p.tol = tol;
    int rc = BDDC_OK;
    auto stage = [&](const double* src, size_t n, double** buf, bool copy_in) -> const double* {
        if (is_device_ptr(src)) return src;
        if (!*buf && cudaMalloc((void**)buf, n * sizeof(double)) != cudaSuccess) { rc = BDDC_E_OOM; return nullptr; }
        if (std::find(h->allocs.begin(), h->allocs.end(), (void*)*buf) == h->allocs.end()) h->allocs.push_back(*buf);
        if (copy_in) cudaMemcpyAsync(*buf, src, n * sizeof(double), cudaMemcpyHostToDevice, st);
        return *buf;
    };
    p.f_in = stage(f, ncell, &h->d_f, true);
    p.bc_in = stage(bc_value, nface, &h->d_bc, true);
    const bool flux_dev = is_device_ptr(flux), p_dev = is_device_ptr(pressure);
    p.flux_out = flux_dev ? flux : const_cast<double*>(stage(flux, nface, &h->d_flux, false));
    p.p_out = p_dev ? pressure : const_cast<double*>(stage(pressure, ncell, &h->d_p, false));
    if (rc) return set_err(h, rc, "staging buffers");
    cudaMemsetAsync(p.flux_out, 0, nface * sizeof(double), st);
    cudaMemsetAsync(p.st, 0, sizeof(InstState) * h->n_inst, st);
    cudaMemsetAsync(p.gsync, 0, sizeof(GridSync), st);
    cudaMemcpyAsync(p.n_active, &h->n_inst, sizeof(int), cudaMemcpyHostToDevice, st);
    void* args[] = {&p};
    const void* kfn = h->precision == BDDC_PREC_FP32 ? (const void*)bddc_solve_kernel<float>
                                                     : (const void*)bddc_solve_kernel<double>;
    cudaEventRecord(h->ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel(kfn, dim3(h->grid), dim3(kThreads), args, h->smem, st);
    cudaEventRecord(h->ev1, st);
    if (e != cudaSuccess) return set_err(h, BDDC_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    if (!flux_dev) cudaMemcpyAsync(flux, p.flux_out, nface * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!p_dev) cudaMemcpyAsync(pressure, p.p_out, ncell * sizeof(double), cudaMemcpyDeviceToHost, st);
    std::vector<InstState> hs(h->n_inst);
    GridSync gs;
    const int64_t H = (int64_t)h->n_inst * (h->maxit + 1);
    std::vector<double> ha(H), hb(H);
    cudaMemcpyAsync(hs.data(), p.st, sizeof(InstState) * h->n_inst, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&gs, p.gsync, sizeof(GridSync), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(ha.data(), p.alpha_hist, sizeof(double) * H, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hb.data(), p.beta_hist, sizeof(double) * H, cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(h, BDDC_E_CUDA, std::string("solve: ") + cudaGetErrorString(e));
    cudaEventElapsedTime(&h->last_ms, h->ev0, h->ev1);
    if (gs.error) return set_err(h, BDDC_E_TIMEOUT, "grid barrier wait exceeded its limit");
    int ret = BDDC_OK;
    double total_it = 0.0;
    int max_it = 0;
    for (int b = 0; b < h->n_inst; ++b) {
        bddc_stats& S = h->stats[b];
        S.iterations = hs[b].iterations;
        S.status = hs[b].done ? hs[b].status : BDDC_E_TIMEOUT;
        S.relres = hs[b].relres;
        // Lanczos estimate from the CG coefficients (Sec. 5)
        const int m = S.iterations;
        S.kappa = 1.0;
        if (m > 0) {
            std::vector<double> dd(m), ee(std::max(m - 1, 1));
            const double* al = &ha[(size_t)b * (h->maxit + 1)];
            const double* be = &hb[(size_t)b * (h->maxit + 1)];
            for (int k = 0; k < m; ++k) {
                dd[k] = 1.0 / al[k] + (k > 0 ? be[k] / al[k - 1] : 0.0);
                if (k + 1 < m) ee[k] = std::sqrt(be[k + 1]) / al[k];
            }
            double lmin, lmax;
            tridiag_extremes(m, dd.data(), ee.data(), &lmin, &lmax);
            S.kappa = lmax / lmin;
        }
        if (iterations) {
            if (is_device_ptr(iterations)) cudaMemcpy(iterations + b, &S.iterations, sizeof(int), cudaMemcpyHostToDevice);
            else iterations[b] = S.iterations;
        }
        if (S.status != BDDC_OK && ret == BDDC_OK) ret = S.status;
        total_it += m;
        max_it = std::max(max_it, m);
    }
    // work of the kernel: every instance runs its own iterations; the
    // persistent loop streams only active instances' operators
    h->last_bytes = h->bytes_pre + h->bytes_post + h->bytes_iter * (total_it / std::max(1, h->n_inst));
    if (ret != BDDC_OK) set_err(h, ret, "one or more instances did not converge");
    return ret;
}

int bddc_get_stats(const bddc_handle* h, int instance, bddc_stats* out) {
    if (!h || !out || instance < 0 || instance >= h->n_inst) return BDDC_E_INVALID_ARG;
    *out = h->stats[instance];
    return BDDC_OK;
}

int bddc_last_solve_timing(const bddc_handle* h, double* kernel_ms, double* algorithmic_bytes) {
    if (!h) return BDDC_E_INVALID_ARG;
    if (kernel_ms) *kernel_ms = h->last_ms;
    if (algorithmic_bytes) *algorithmic_bytes = h->last_bytes;
    return BDDC_OK;
}

int bddc_apply_operator(bddc_handle* h, const double* u, const double* p0, double* q) {
    if (!h || !u || !p0 || !q) return BDDC_E_INVALID_ARG;
    if (!is_device_ptr(u) || !is_device_ptr(p0) || !is_device_ptr(q))
        return set_err(h, BDDC_E_INVALID_ARG, "device pointers required");
    Params p = h->prm;
    const int grid = (int)std::min<int64_t>(p.n_sub, 4096);
    k_operator_local<<<grid, kThreads, h->smem, h->stream>>>(p, u, p0);
    const int64_t L = h->P.off_slot.back();
    k_assemble<<<(int)std::min<int64_t>((L + 255) / 256, 4096), 256, 0, h->stream>>>(L, p.ql, p.slot_g, p.slot_partner, q);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? BDDC_OK : set_err(h, BDDC_E_CUDA, cudaGetErrorString(e));
}

int bddc_apply_preconditioner(bddc_handle* h, const double* r, double* z, double* z0) {
    if (!h || !r || !z || !z0) return BDDC_E_INVALID_ARG;
    if (!is_device_ptr(r) || !is_device_ptr(z) || !is_device_ptr(z0))
        return set_err(h, BDDC_E_INVALID_ARG, "device pointers required");
    Params p = h->prm;
    cudaMemsetAsync(p.st, 0, sizeof(InstState) * h->n_inst, h->stream);
    const int grid = (int)std::min<int64_t>(p.n_sub, 4096);
    if (h->precision == BDDC_PREC_FP32) {
        k_precond_restrict<float><<<grid, kThreads, h->smem, h->stream>>>(p, r);
    } else {
        k_precond_restrict<double><<<grid, kThreads, h->smem, h->stream>>>(p, r);
    }
    k_precond_coarse<<<(int)std::min<int64_t>(p.n_cunits, 4096), kThreads, h->smem, h->stream>>>(p);
    if (h->precision == BDDC_PREC_FP32) {
        k_precond_prolong<float><<<grid, kThreads, h->smem, h->stream>>>(p, z0);
    } else {
        k_precond_prolong<double><<<grid, kThreads, h->smem, h->stream>>>(p, z0);
    }
    const int64_t L = h->P.off_slot.back();
    k_assemble<<<(int)std::min<int64_t>((L + 255) / 256, 4096), 256, 0, h->stream>>>(L, p.zl, p.slot_g, p.slot_partner, z);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? BDDC_OK : set_err(h, BDDC_E_CUDA, cudaGetErrorString(e));
}

int bddc_subassembled_apply(int n_sub, const int* ng, const int64_t* slot_offset, const int64_t* S_offset,
                            const double* S, const int* gidx, const int* partner, int64_t n_interface,
                            const double* u, double* q, double* slot_scratch, void* stream) {
    if (n_sub <= 0 || !ng || !slot_offset || !S_offset || !S || !gidx || !partner || !u || !q || !slot_scratch ||
        n_interface <= 0)
        return BDDC_E_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t n_slots = 0;
    if (cudaMemcpy(&n_slots, slot_offset + n_sub, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BDDC_E_CUDA;
    std::vector<int> hng(n_sub);
    if (cudaMemcpy(hng.data(), ng, sizeof(int) * n_sub, cudaMemcpyDeviceToHost) != cudaSuccess) return BDDC_E_CUDA;
    for (int v : hng)
        if (v < 0 || v > 1024) return BDDC_E_INVALID_ARG;
    k_subassembled_local<<<std::min(n_sub, 4096), kThreads, 0, st>>>(n_sub, ng, slot_offset, S_offset, S, gidx, u,
                                                                     slot_scratch);
    k_assemble<<<(int)std::min<int64_t>((n_slots + 255) / 256, 4096), 256, 0, st>>>(n_slots, slot_scratch, gidx, partner, q);
    return cudaGetLastError() == cudaSuccess ? BDDC_OK : BDDC_E_CUDA;
}

}  // extern "C"

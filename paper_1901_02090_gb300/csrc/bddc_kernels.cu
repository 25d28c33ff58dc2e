// GB300 (sm_103a) kernels and C ABI of the BDDC solver.
//
// The solve is one persistent cooperative kernel (bddc_solve_kernel) per
// batch of instances.  Its phases follow Algorithm 1 of the paper:
//   Step 1  coarse right-hand side, coarse solve, u_0 = E w_0;
//   Step 2  local residuals S u_0 + G f of the subdomain problems, giving the
//           reduced right-hand side f* of eqs. (corr-reduced-1/2);
//   Step 3  CG on the pairs (w_hat, p_0) with the BDDC preconditioner of
//           Algorithm 2; per iteration four phases:
//             DIROP   d = z + beta d, q = S d + B_0^T d_p, (d, q) -> alpha
//             UPDATE  x += alpha d, r -= alpha q, (r, r), weighted
//                     restriction, subdomain correction F r, Psi^T r
//             COARSE  coarse solve
//             PROLONG z = E (Psi w_c + F r), (r, z) -> convergence test
//                     and beta of the next iteration
//           The scalar step of each instance (alpha, the test, beta) is
//           taken once, by the warp that completes the instance's partial
//           inner products.
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
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bddc_internal.hpp"
#include "bddc_kernels.cuh"
#include "dense.hpp"

namespace bddc {

#include "bddc_cache.cuh"

// ---- small device helpers --------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool slot_owner(int slot, int partner) { return partner < 0 || slot < partner; }

// warp-uniform read of an instance's done flag (the owner warp may set it
// while other warps are in the same phase)
__device__ __forceinline__ int inst_done(const Params& p, int b) {
    int f = 0;
    if ((threadIdx.x & 31) == 0) f = __ldcg(&p.st[b].done);
    return __shfl_sync(0xffffffffu, f, 0);
}

// block-uniform read, for the CTA-level coarse phase
__device__ int inst_done_block(const Params& p, int b) {
    __shared__ int flag;
    __syncthreads();
    if (threadIdx.x == 0) flag = __ldcg(&p.st[b].done);
    __syncthreads();
    return flag;
}

// fixed-order sum of part[s0..s1) by one warp (every lane gets the result)
__device__ __forceinline__ double range_sum(const double* part, int64_t s0, int64_t s1) {
    double v = 0.0;
    for (int64_t s = s0 + (threadIdx.x & 31); s < s1; s += 32) v += __ldcg(part + s);
    return warp_sum(v);
}

// ---- per-instance CG scalars ----------------------------------------------------
// Each subdomain warp stores its partial of an inner product and counts its
// arrival with an acquire-release atomic.  The warp whose arrival completes
// the instance sums the instance's partials in a fixed order (range_sum) and
// takes the instance's scalar step of CG once: at the end of PROLONG the
// convergence test of iteration k and its beta (from rr = (r, r) of the last
// residual update and rz = (r, z)), at the end of DIROP alpha = rho / (d, q).
// The warps of the next phase read the published values instead of each
// re-summing the partials and repeating the FP64 arithmetic.  The completing
// warp resets the count for the next use (after the next grid barrier).
enum : int { kCtrRR = 0, kCtrRZ = 1, kCtrDQ = 2, kCounters = 3 };
enum : int { kTotRR = 0, kTotRZ = 1, kTotDQ = 2, kTotA1 = 3, kTotA2 = 4, kTotals = 5 };
constexpr double kRhoFluxConverged = 1e-24;

__device__ __forceinline__ int arrive_acq_rel(int* cnt, int n = 1) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(cnt), "r"(n) : "memory");
    return old;
}

// convergence test of iteration k (Sec. 6: relative residual, with the
// rounding floor and the converged-flux test of (r, z)); beta_k on
// continuation, the final bookkeeping otherwise.  Whole warp.
__device__ void cg_decide(const Params& p, int b, int k, double rz, bool fp64_correction) {
    const int l = threadIdx.x & 31;
    const int64_t s0 = p.inst_s0[b], s1 = p.inst_s1[b];
    const double* tot = p.inst_tot + (int64_t)b * kTotals;
    const int64_t hb = (int64_t)b * (p.maxit + 1);
    const double rr = __ldcg(tot + kTotRR);
    double r0, floor_, rho0;
    if (k == 0) {
        r0 = sqrt(rr);
        floor_ = 1e-14 * (sqrt(__ldcg(tot + kTotA1)) + sqrt(__ldcg(tot + kTotA2)));
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
        // M is positive semi-definite: (r, z) <= 0 at the start is a rounded
        // zero, i.e. r lies in range(B_0^T) and the flux is already exact
        if (nr <= floor_ || rz <= 0.0) status = BDDC_OK;
        else if (!(rz == rz)) status = BDDC_E_BREAKDOWN;
    } else {
        if (relres <= p.tol || nr <= floor_ || rz <= kRhoFluxConverged * rho0) status = BDDC_OK;
        else if (!(rz > 0.0)) status = BDDC_E_BREAKDOWN;
        else if (k >= p.maxit) status = BDDC_E_NOT_CONVERGED;
    }
    if (l == 0) {
        if (k == 0) {
            p.st[b].r0 = r0;
            p.st[b].floor = floor_;
            p.st[b].rho0 = rho0;
        }
        p.rho_hist[hb + k] = rz;
        if (status == -100) p.beta_hist[hb + k] = (k == 0) ? 0.0 : rz / __ldcg(p.rho_hist + hb + k - 1);
    }
    if (status != -100) {
        // FP64 path: last coarse pressure correction x_p += z_p from the
        // final residual (the mixed path does it in FP64 after the loop)
        if (fp64_correction)
            for (int64_t t = s0 + l; t < s1; t += 32) p.xp[t] = __ldcg(p.xp + t) + __ldcg(p.zp + t);
        __syncwarp();
        if (l == 0) {
            p.st[b].status = status;
            p.st[b].iterations = k;
            p.st[b].relres = relres;
            p.st[b].fin = phase_index(k, kPhProlong) + 1;
            __threadfence();
            p.st[b].done = 1;
            atomicSub(p.n_active, 1);
        }
    }
    __syncwarp();
}

// alpha_k = rho_k / (d, q), or breakdown when (d, q) <= 0.  Lane 0.
__device__ void cg_alpha(const Params& p, int b, int k, double dq) {
    if ((threadIdx.x & 31) != 0) return;
    const int64_t hb = (int64_t)b * (p.maxit + 1);
    if (!(dq > 0.0)) {
        p.st[b].status = BDDC_E_BREAKDOWN;
        p.st[b].iterations = k;
        p.st[b].relres = -1.0;
        p.st[b].fin = phase_index(k, kPhDirop) + 1;
        __threadfence();
        p.st[b].done = 1;
        atomicSub(p.n_active, 1);
    } else {
        p.alpha_hist[hb + k] = __ldcg(p.rho_hist + hb + k) / dq;
    }
}

// count the arrival of n units of instance b whose partials of kind ctr
// this warp has stored (subdomains; operator-apply units for kCtrDQ); the
// completing warp publishes the total (the partials summed in unit order)
// and takes the scalar step.  A warp counts all its consecutive units of an
// instance with one atomic (it usually holds several per phase).
__device__ void publish_total(const Params& p, int b, int n, int ctr, int k = 0, bool with_a = false,
                              bool fp64_correction = false) {
    const bool du = ctr == kCtrDQ;
    const int64_t s0 = du ? p.inst_du0[b] : p.inst_s0[b], s1 = du ? p.inst_du0[b + 1] : p.inst_s1[b];
    int* cnt = p.inst_cnt + (int64_t)b * kCounters + ctr;
    int last = 0;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) last = arrive_acq_rel(cnt, n) == (int)(s1 - s0) - n;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    const double* part = ctr == kCtrRR ? p.part_rr : (ctr == kCtrRZ ? p.part_rz : p.part_dq);
    const double v = range_sum(part, s0, s1);
    double a1 = 0.0, a2 = 0.0;
    if (with_a) {
        a1 = range_sum(p.part_a1, s0, s1);
        a2 = range_sum(p.part_a2, s0, s1);
    }
    if ((threadIdx.x & 31) == 0) {
        double* tot = p.inst_tot + (int64_t)b * kTotals;
        tot[ctr == kCtrRR ? kTotRR : (ctr == kCtrRZ ? kTotRZ : kTotDQ)] = v;
        if (with_a) {
            tot[kTotA1] = a1;
            tot[kTotA2] = a2;
        }
        *cnt = 0;
    }
    __syncwarp();
    if (ctr == kCtrRZ) cg_decide(p, b, k, v, fp64_correction);
    else if (ctr == kCtrDQ) cg_alpha(p, b, k, v);
}

// grid-wide barrier with a wait bounded in time (limit_ns of %globaltimer);
// past the limit the CTA sets the error flag and returns false, as does
// every CTA that finds the flag set, so the kernel ends and the host reads
// BDDC_E_TIMEOUT with the context intact
__device__ bool grid_barrier(GridSync* gs, long long limit_ns = kBarrierWaitNs) {
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
            long long t0, t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (unsigned int spins = 1; *vgen == g0; ++spins) {
                __nanosleep(32);
                if ((spins & 255) == 0) {
                    if (*(volatile int*)&gs->error) { ok = 0; break; }
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (t - t0 > limit_ns) { ok = 0; break; }
                }
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

// grid barrier that also records, on CTA 0, the phase that just ended and
// the global timer (ns) when the barrier released
__device__ __forceinline__ bool phase_end(const Params& p, int phase, int& nts) {
    const bool ok = grid_barrier(p.gsync);
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.tstamp && nts < p.tstamp_cap) {
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        p.tstamp[2 * nts] = phase;
        p.tstamp[2 * nts + 1] = t;
        ++nts;
    }
    return ok;
}

// contiguous chunk of U units for this CTA / this warp
__device__ __forceinline__ void cta_range(int64_t U, int64_t& a, int64_t& b) {
    a = (U * (int64_t)blockIdx.x) / gridDim.x;
    b = (U * ((int64_t)blockIdx.x + 1)) / gridDim.x;
}
__device__ __forceinline__ void warp_range(int64_t U, int64_t& a, int64_t& b) {
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    a = (U * w) / W;
    b = (U * (w + 1)) / W;
}
// this warp's contiguous range of subdomains, balanced by work: the host
// splits the subdomains at equal fractions of the summed cost n_Gamma^2 + C
// (S and F, plus the fixed latency C of a unit: 4096, or the autotuner's
// choice), so a warp drawn several large subdomains of an uneven partition
// does not set the length of a phase
__device__ __forceinline__ void sub_range(const Params& p, int64_t& a, int64_t& b) {
    const int64_t w = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    a = p.warp_sub0[w];
    b = p.warp_sub0[w + 1];
}

// ---- precisions ------------------------------------------------------------------
struct PrecFP64 {
    using S_t = double;
    using F_t = double;
    static constexpr bool kMixed = false;
    static constexpr bool kFull = false;
};
// FP64 with the operator in its full-space form (BDDC_FORM_FULL)
struct PrecFP64Full : PrecFP64 {
    static constexpr bool kFull = true;
};
struct PrecMixed {
    using S_t = float2;   // the operator as an FP32 pair (48 significant bits)
    using F_t = float;
    static constexpr bool kMixed = true;
    static constexpr bool kFull = false;
};

// Per-warp shared-memory slice: the staged input vector in FP64 and as an
// FP32 pair (hi + lo), a second input vector for the Step-2 / post maps, and
// the subdomain's coarse values.
struct WarpSm {
    double* x;
    float* xh;
    float* xl;
    double* xin;
    double* wcs;
    double* tsum;  // per net-flux row sums (mixed path); the full form's extension follows
};
struct CtaSm {
    double* rhs;  // staged coarse right-hand side (CTA-level)
    WarpSm w;
};
// kExt: the warp areas include the full form's extension (max_ext doubles)
template <bool kExt = false>
__device__ __forceinline__ CtaSm carve(const Params& p, double* base) {
    CtaSm c;
    c.rhs = base;
    const int warp = threadIdx.x >> 5;
    const int per_warp = 2 * p.max_ng + p.max_in_post + 2 * (p.max_m + 1) + (kExt ? p.max_ext : 0);  // in doubles
    double* wb = base + p.max_ncn + (int64_t)warp * per_warp;
    c.w.x = wb;
    c.w.xh = reinterpret_cast<float*>(wb + p.max_ng);
    c.w.xl = c.w.xh + p.max_ng;
    c.w.xin = wb + 2 * p.max_ng;
    c.w.wcs = c.w.xin + p.max_in_post;
    c.w.tsum = c.w.wcs + p.max_m + 1;
    return c;
}

// Active-instance snapshot of the current CG iteration (p.act_n > 0), after
// the warp areas of the persistent kernel's shared memory: exclusive prefix
// sums over the instances of the active subdomains (act_sub) and of the
// active coarse units (act_cu = act_sub + n_inst + 1), n_inst + 1 each.  The
// address is formed where it is used, so that no register holds it across
// the phases (the kernel runs at its register cap).
template <bool kExt>
__device__ __forceinline__ int* act_area(const Params& p, double* base) {
    const int per_warp = 2 * p.max_ng + p.max_in_post + 2 * (p.max_m + 1) + (kExt ? p.max_ext : 0);
    return reinterpret_cast<int*>(base + p.max_ncn + (int64_t)kWarps * per_warp);
}
// set by active_snapshot: the current CG iteration rebalances its phases
__shared__ int g_partial_sh;

// Snapshot of the instances active in CG phase P (fin = 0 or fin > P), per
// CTA: exclusive prefix sums over the instances of their subdomain counts
// and coarse-unit counts (0 for inactive instances).  Whole CTA; returns
// the number of active subdomains.  Every CTA computes the same snapshot.
__device__ int64_t active_snapshot(const Params& p, int* act_sub, int P) {
    int* act_cu = act_sub + p.act_n + 1;
    const int n = p.act_n;
    const int per = (n + kThreads - 1) / kThreads;
    const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
    // fin is read once: bit t of `on` is instance i0 + t (per <= 16 for kActMaxInst)
    int cs = 0, cu = 0;
    unsigned on = 0u;
    for (int b = i0; b < i1; ++b) {
        const int f = __ldcg(&p.st[b].fin);
        if (f == 0 || f > P) {
            on |= 1u << (b - i0);
            cs += (int)(p.inst_s1[b] - p.inst_s0[b]);
            cu += (int)(p.inst_cu0[b + 1] - p.inst_cu0[b]);
        }
    }
    // block exclusive scan of (cs, cu): warp scans, then the warp totals
    __shared__ int wtot[2 * kWarps];
    const int l = threadIdx.x & 31, wi = threadIdx.x >> 5;
    int xs = cs, xu = cu;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ys = __shfl_up_sync(0xffffffffu, xs, o), yu = __shfl_up_sync(0xffffffffu, xu, o);
        if (l >= o) {
            xs += ys;
            xu += yu;
        }
    }
    __syncthreads();
    if (l == 31) {
        wtot[wi] = xs;
        wtot[kWarps + wi] = xu;
    }
    __syncthreads();
    int bs = 0, bu = 0;
    for (int q = 0; q < wi; ++q) {
        bs += wtot[q];
        bu += wtot[kWarps + q];
    }
    int es = bs + xs - cs, eu = bu + xu - cu;  // exclusive prefix of this thread's first instance
    for (int b = i0; b < i1; ++b) {
        act_sub[b] = es;
        act_cu[b] = eu;
        if (on & (1u << (b - i0))) {
            es += (int)(p.inst_s1[b] - p.inst_s0[b]);
            eu += (int)(p.inst_cu0[b + 1] - p.inst_cu0[b]);
        }
    }
    if (threadIdx.x == kThreads - 1) {
        int ts = 0, tu = 0;
        for (int q = 0; q < kWarps; ++q) {
            ts += wtot[q];
            tu += wtot[kWarps + q];
        }
        act_sub[n] = ts;
        act_cu[n] = tu;
        g_partial_sh = ts > 0 && ts < p.n_sub;
    }
    __syncthreads();
    return act_sub[n];
}

// the instance b with pre[b] <= x < pre[b + 1] (pre non-decreasing, n + 1 entries)
__device__ __forceinline__ int act_find(const int* pre, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// stage x[0..n) as FP32 (hi only: inputs of the FP32 operators)
__device__ __forceinline__ void split_hi(WarpSm w, int n) {
    for (int k = threadIdx.x & 31; k < n; k += 32) w.xh[k] = __double2float_rn(w.x[k]);
    __syncwarp();
}

// stage x[0..n) from the warp's x into the FP32 pair representation
__device__ __forceinline__ void split_pairs(WarpSm w, int n) {
    for (int k = threadIdx.x & 31; k < n; k += 32) {
        const double v = w.x[k];
        const float h = __double2float_rn(v);
        w.xh[k] = h;
        w.xl[k] = __double2float_rn(v - (double)h);
    }
    __syncwarp();
}

#include "bddc_dd.cuh"
#include "bddc_gemv.cuh"

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float2 v) { return dd_dbl(v); }

// restriction rc_a = sum_k P[a*ng + k] x[k]: lane per row a, walking its
// contiguous row (consecutive loads of one lane share cache lines); all
// loads are independent, so one pass costs about one memory latency
__device__ __forceinline__ void restrict_rows(const double* __restrict__ P, int m, int ng, const WarpSm w, double* out) {
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        const double* row = P + (int64_t)a * ng;
        double a0 = 0.0, a1 = 0.0;
        int k = 0;
#pragma unroll 4
        for (; k + 1 < ng; k += 2) {
            a0 = fma(__ldg(row + k), w.x[k], a0);
            a1 = fma(__ldg(row + k + 1), w.x[k + 1], a1);
        }
        if (k < ng) a0 = fma(__ldg(row + k), w.x[k], a0);
        out[a] = a0 + a1;
    }
}
__device__ __forceinline__ void restrict_rows(const float* __restrict__ P, int m, int ng, const WarpSm w, double* out,
                                              const double* add = nullptr) {
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        const float* row = P + (int64_t)a * ng;
        float a0 = 0.0f, a1 = 0.0f;
        int k = 0;
#pragma unroll 4
        for (; k + 1 < ng; k += 2) {
            a0 = fmaf(__ldg(row + k), w.xh[k], a0);
            a1 = fmaf(__ldg(row + k + 1), w.xh[k + 1], a1);
        }
        if (k < ng) a0 = fmaf(__ldg(row + k), w.xh[k], a0);
        out[a] = (double)(a0 + a1) + (add ? add[a] : 0.0);
    }
}

// prolongation value for output k: sum_a P[a*ng + k] wcs[a]
__device__ __forceinline__ double prolong_out(const double* __restrict__ P, int m, int ng, const WarpSm w, int k) {
    double acc = 0.0;
    for (int a = 0; a < m; ++a) acc = fma(__ldg(P + (int64_t)a * ng + k), w.wcs[a], acc);
    return acc;
}
__device__ __forceinline__ double prolong_out(const float* __restrict__ P, int m, int ng, const WarpSm w, int k) {
    float acc = 0.0f;
    for (int a = 0; a < m; ++a) acc = fmaf(__ldg(P + (int64_t)a * ng + k), (float)w.wcs[a], acc);
    return (double)acc;
}

// Mixed path.  P_Z removes the net flux of a local vector through each face
// (a symmetric projection); the FP32 operators are applied as P_Z F P_Z and
// Psi_0 + P_Z Psi, where Psi_0 puts the unit net flux of a face-constraint
// column uniformly on the face's dofs.  In exact arithmetic these equal F and
// Psi; in rounded arithmetic restriction and prolongation stay transposes
// and the preconditioner output keeps exact face net fluxes, so it stays
// balanced (Sec. 3) to FP64 rounding.
//
// t[a] = (sum over the dofs of net-flux row a of coef * v) / (dofs of a),
// lane per row; 0 for adaptive rows
__device__ __forceinline__ void face_sums(const Params& p, int64_t s, const double* v, double* t) {
    const int m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        const int na = p.cslot_n[co + a];
        double acc = 0.0;
        if (na > 0) {
            const int64_t fs = so + p.cslot_fstart[co + a];
#pragma unroll 4
            for (int q = 0; q < na; ++q) acc += __ldg(p.slot_fcoefp + fs + q) * v[__ldg(p.slot_fperm + fs + q)];
            acc /= (double)na;
        }
        t[a] = acc;
    }
    __syncwarp();
}
// v <- P_Z v
__device__ __forceinline__ void remove_face_flux(const Params& p, int64_t s, double* v, const double* t) {
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    for (int k = threadIdx.x & 31; k < ng; k += 32) v[k] -= p.slot_coef[so + k] * t[p.slot_fcs[so + k]];
    __syncwarp();
}
// v <- P_Z v + Psi_0 wcs
__device__ __forceinline__ void set_face_flux(const Params& p, int64_t s, double* v, double* t, const double* wcs) {
    const int m = p.sub_m[s];
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    for (int a = threadIdx.x & 31; a < m; a += 32) {
        const int na = p.cslot_n[co + a];
        if (na > 0) t[a] = wcs[a] / (double)na - t[a];
    }
    __syncwarp();
    for (int k = threadIdx.x & 31; k < ng; k += 32) v[k] += p.slot_coef[so + k] * t[p.slot_fcs[so + k]];
    __syncwarp();
}

__device__ __forceinline__ void stage_wc(const Params& p, int64_t s, const double* wc_b, WarpSm w) {
    const int m = p.sub_m[s];
    const int64_t co = p.off_cslot[s];
    for (int a = threadIdx.x & 31; a < m; a += 32) w.wcs[a] = __ldcg(wc_b + p.cslot_c[co + a]);
    __syncwarp();
}

// subdomain correction and coarse restriction of the weighted residual in
// w.x: yl = F x, rcl = Psi^T x (Algorithm 2 steps 1-2, local parts)
template <class PR>
__device__ void restrict_apply(const Params& p, int64_t s, WarpSm w) {
    using F_t = typename PR::F_t;
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const F_t* F = reinterpret_cast<const F_t*>(p.F) + p.off_F[s];
    const F_t* P = reinterpret_cast<const F_t*>(p.P) + p.off_P[s];
    if constexpr (PR::kMixed) {
        // rc = Psi_0^T r + Psi^T P_Z r ; y = P_Z F P_Z r
        face_sums(p, s, w.x, w.tsum);
        remove_face_flux(p, s, w.x, w.tsum);
        split_hi(w, ng);
        restrict_rows(P, m, ng, w, p.rcl + co, w.tsum);  // tsum is 0 on adaptive rows
        __syncwarp();
        gemv_warp(F, ng, w, [&](int k, double v) { w.xin[k] = v; });
        __syncwarp();
        face_sums(p, s, w.xin, w.tsum);
        remove_face_flux(p, s, w.xin, w.tsum);
        for (int k = threadIdx.x & 31; k < ng; k += 32) p.yl[so + k] = w.xin[k];
    } else {
        gemv_warp(F, ng, w, [&](int k, double v) { p.yl[so + k] = v; });
        restrict_rows(P, m, ng, w, p.rcl + co);
    }
    __syncwarp();
}

// ---- phases (warp per subdomain unless noted) --------------------------------------
template <class PR>
__device__ void ph_step1(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int l = threadIdx.x & 31;
    for (int k = l; k < ng; k += 32) {
        const int gi = p.slot_g[so + k];
        const double sg = p.g_bsign[gi];
        const double gv = sg != 0.0 ? sg * p.bc_in[p.g_fid[gi]] : 0.0;
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.g[gi] = gv;
        w.x[k] = p.slot_w[so + k] * gv;
    }
    __syncwarp();
    // Step 1 right-hand side <g, E psi> with the FP64 coarse basis
    restrict_rows(p.P64 + p.off_P[s], m, ng, w, p.rcl + co);
    double v = 0.0;
    const int64_t cb = p.off_cell[s];
    for (int r = l; r < nc; r += 32) v += -p.f_in[p.cell_gid[cb + r]];
    v = warp_sum(v);
    if (l == 0) p.prhs[s] = p.sub_d[s] * p.inst_vol[b] * v;
    __syncwarp();
}

// coarse solve rows (CTA per unit): wc = Kinv * rhs; rhs flux part from the
// coarse slots, pressure part the Step-1 right-hand side or zero
template <class PR>
__device__ void ph_coarse(const Params& p, int64_t u, bool step1, double* rhs, int& staged) {
    using K_t = typename std::conditional<PR::kMixed, float2, double>::type;
    const int b = p.cunit_inst[u];
    if (!step1 && inst_done_block(p, b)) return;
    const int64_t ncn = p.inst_ncn[b], ncf = p.inst_ncf[b], coff = p.inst_coff[b];
    const int64_t cfo = p.inst_cfoff[b];
    const int64_t ncols = step1 ? ncn : ncf;
    float2* rhs2 = reinterpret_cast<float2*>(rhs);  // mixed: the rhs as FP32 pairs
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
            if constexpr (PR::kMixed) {
                const float hi = __double2float_rn(v);
                rhs2[c] = make_float2(hi, __double2float_rn(v - (double)hi));
            } else {
                rhs[c] = v;
            }
        }
        __syncthreads();
        staged = b;
    }
    const K_t* K = reinterpret_cast<const K_t*>(p.Kinv) + p.inst_kinv_off[b];
    const uint64_t pol = l2_stream_policy();
    const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int64_t r0 = p.cunit_row0[u];
    const int64_t r1 = (r0 + p.coarse_rows < ncn) ? r0 + p.coarse_rows : ncn;
    for (int64_t row = r0 + wi; row < r1; row += kWarps) {
        const K_t* kr = K + row * ncn;
        double acc;
        if constexpr (PR::kMixed) {
            float sh = 0.0f, sl = 0.0f;
            for (int64_t c = l; c < ncols; c += 32) {
                const float2 a = ld_hint(kr + c, pol);
                const float2 xv = rhs2[c];
                const float xh = xv.x, xl = xv.y;
                const float pr = __fmul_rn(a.x, xh);
                float e = __fmaf_rn(a.x, xh, -pr);
                e = __fmaf_rn(a.x, xl, e);
                e = __fmaf_rn(a.y, xh, e);
                const float t = __fadd_rn(sh, pr);
                const float bp = __fsub_rn(t, sh);
                const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(pr, bp));
                sh = t;
                sl = __fadd_rn(sl, __fadd_rn(err, e));
            }
            acc = (double)sh + (double)sl;
        } else {
            acc = 0.0;
            int64_t c = l;
            for (; c + 7 * 32 < ncols; c += 8 * 32) {
                double A[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) A[t] = ld_hint(reinterpret_cast<const double*>(kr) + c + 32 * t, pol);
#pragma unroll
                for (int t = 0; t < 8; ++t) acc = fma(A[t], rhs[c + 32 * t], acc);
            }
            for (; c < ncols; c += 32) acc = fma(ld_hint(reinterpret_cast<const double*>(kr) + c, pol), rhs[c], acc);
        }
        acc = warp_sum(acc);
        if (l == 0) p.wc[coff + row] = acc;
    }
}

template <class PR>
__device__ void ph_u0(const Params& p, int64_t s, WarpSm w) {
    using F_t = typename PR::F_t;
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s];
    stage_wc(p, s, p.wc + p.inst_coff[b], w);
    const F_t* P = reinterpret_cast<const F_t*>(p.P) + p.off_P[s];
    for (int k = threadIdx.x & 31; k < ng; k += 32) w.xin[k] = prolong_out(P, m, ng, w, k);
    __syncwarp();
    if constexpr (PR::kMixed) {
        face_sums(p, s, w.xin, w.tsum);
        set_face_flux(p, s, w.xin, w.tsum, w.wcs);
    }
    for (int k = threadIdx.x & 31; k < ng; k += 32) p.tl[so + k] = p.slot_w[so + k] * w.xin[k];
    __syncwarp();
}

// Step 2 local residual r_G = S u_0 + G_pre f (stored in ql)
template <class PR>
__device__ void ph_step2(const Params& p, int64_t s, WarpSm w) {
    using S_t = typename PR::S_t;
    const int ng = p.sub_ng[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], cb = p.off_cell[s];
    const int l = threadIdx.x & 31;
    for (int k = l; k < ng; k += 32) {
        const int pt = p.slot_partner[so + k];
        const double u = __ldcg(p.tl + so + k) + (pt >= 0 ? __ldcg(p.tl + pt) : 0.0);
        if (slot_owner((int)(so + k), pt)) p.u0[p.slot_g[so + k]] = u;
        w.x[k] = u;
    }
    int nz = 0;
    for (int r = l; r < nc; r += 32) {
        const double fv = p.f_in[p.cell_gid[cb + r]];
        w.xin[r] = fv;
        nz |= (fv != 0.0);
    }
    const int nsrc = __any_sync(0xffffffffu, nz) ? nc : 0;  // f = 0: G_pre f vanishes exactly
    __syncwarp();
    if constexpr (PR::kMixed) split_pairs(w, ng);
    const S_t* S = reinterpret_cast<const S_t*>(p.S) + p.off_S[s];
    const double* G = p.Gpre + p.off_Gpre[s];
    gemv_warp(S, ng, w, [&](int k, typename GAcc<S_t>::value_type y) {
        double acc = to_double(y);
        for (int r = 0; r < nsrc; ++r) acc = fma(__ldg(G + (int64_t)r * ng + k), w.xin[r], acc);
        p.ql[so + k] = acc;
    });
    __syncwarp();
}

// f* = g - sum_i R_i^T r_G,i ; r_0 = f*, x_0 = 0 ; then restrict r_0
template <class PR>
__device__ void ph_fstar(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    const int l = threadIdx.x & 31;
    double rr = 0.0, a1 = 0.0, a2 = 0.0;
    for (int k = l; k < ng; k += 32) {
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
        w.x[k] = wr;
        p.rl[so + k] = wr;
    }
    rr = warp_sum(rr);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (l == 0) {
        p.part_rr[s] = rr;
        p.part_a1[s] = a1;
        p.part_a2[s] = a2;
        p.xp[s] = 0.0;
        p.dp0[s] = 0.0;
        p.dp1[s] = 0.0;
    }
    __syncwarp();
    publish_total(p, p.sub_inst[s], 1, kCtrRR, 0, true);
    restrict_apply<PR>(p, s, w);
}

// The CG phases store their partials and return false for an instance that
// is done; the caller counts the arrivals (publish_total).
template <class PR>
__device__ bool ph_prolong(const Params& p, int64_t s, WarpSm w) {
    using F_t = typename PR::F_t;
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s];
    const double* wcb = p.wc + p.inst_coff[b];
    stage_wc(p, s, wcb, w);
    const F_t* P = reinterpret_cast<const F_t*>(p.P) + p.off_P[s];
    for (int k = threadIdx.x & 31; k < ng; k += 32) w.xin[k] = prolong_out(P, m, ng, w, k);
    __syncwarp();
    if constexpr (PR::kMixed) {
        face_sums(p, s, w.xin, w.tsum);
        set_face_flux(p, s, w.xin, w.tsum, w.wcs);
    }
    for (int k = threadIdx.x & 31; k < ng; k += 32) w.xin[k] += __ldcg(p.yl + so + k);
    __syncwarp();
    double rz = 0.0;
    for (int k = threadIdx.x & 31; k < ng; k += 32) {
        const double z = w.xin[k];
        p.zl[so + k] = p.slot_w[so + k] * z;
        rz += __ldcg(p.rl + so + k) * z;
    }
    rz = warp_sum(rz);
    if ((threadIdx.x & 31) == 0) {
        p.part_rz[s] = rz;
        p.zp[s] = __ldcg(wcb + p.inst_ncf[b] + p.sub_local[s]);
    }
    __syncwarp();
    return true;
}

// direction update d = z + beta d and operator apply q = S d + B_0^T d_p,
// for the outputs [ob, oe) of operator-apply unit u of subdomain s (the unit
// with ob = 0 also stores the subdomain's new direction)
template <class PR>
__device__ bool ph_dirop(const Params& p, int64_t u, int64_t s, int ob, int oe, int k, WarpSm w) {
    using S_t = typename PR::S_t;
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int l = threadIdx.x & 31;
    const double beta = __ldcg(p.beta_hist + (int64_t)b * (p.maxit + 1) + k);
    double* dold = (k & 1) ? p.dbuf0 : p.dbuf1;
    double* dnew = (k & 1) ? p.dbuf1 : p.dbuf0;
    double* dpold = (k & 1) ? p.dp0 : p.dp1;
    double* dpnew = (k & 1) ? p.dp1 : p.dp0;
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    for (int kk = l; kk < ng; kk += 32) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        const double z = __ldcg(p.zl + so + kk) + (pt >= 0 ? __ldcg(p.zl + pt) : 0.0);
        const double dn = (k == 0) ? z : z + beta * __ldcg(dold + gi);
        if (ob == 0 && slot_owner((int)(so + kk), pt)) dnew[gi] = dn;
        w.x[kk] = dn;
    }
    const double dpn = (k == 0) ? __ldcg(p.zp + s) : __ldcg(p.zp + s) + beta * __ldcg(dpold + s);
    if (l == 0 && ob == 0) dpnew[s] = dpn;
    __syncwarp();
    if constexpr (PR::kMixed) split_pairs(w, ng);
    const S_t* S = reinterpret_cast<const S_t*>(p.S) + p.off_S[s];
    double dq = 0.0;
    gemv_warp_range(S, ng, ob, oe, w, [&](int kk, typename GAcc<S_t>::value_type y) {
        const double q = to_double(y) + p.slot_dsig[so + kk] * dpn;
        p.ql[so + kk] = q;
        dq += w.x[kk] * q;
    });
    dq = warp_sum(dq);
    if (l == 0) p.part_dq[u] = dq;
    __syncwarp();
    return true;
}

// Full-space form of the same phase (BDDC_FORM_FULL, FP64).  The direction
// d on the interface and its pressure constant p_0 define a vector of the
// full RT0/P0 space: interior fluxes and cell pressures from the discrete
// harmonic extension (the interface columns of the post-correction map
// G_post; cell pressure d_s (p_0 + extension)).  The mixed operator of
// Sec. 2 applied to it has nonzero rows only on the interface faces; each
// such face of the subdomain has one cell K here, and its row is the face's
// row of K's RT0 mass block, h_a^2 / (|K| k_a) (u_e / 3 + u_opp / 6), plus
// +p_K if the face is K's lower face, -p_K if its upper face.  Equal to
// S^i d + d_s sigma p_0 up to rounding (the condensed form).
template <class PR>
__device__ bool ph_dirop_full(const Params& p, int64_t u, int64_t s, int k, WarpSm w) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int l = threadIdx.x & 31;
    const double beta = __ldcg(p.beta_hist + (int64_t)b * (p.maxit + 1) + k);
    double* dold = (k & 1) ? p.dbuf0 : p.dbuf1;
    double* dnew = (k & 1) ? p.dbuf1 : p.dbuf0;
    double* dpold = (k & 1) ? p.dp0 : p.dp1;
    double* dpnew = (k & 1) ? p.dp1 : p.dp0;
    const int ng = p.sub_ng[s], ni = p.sub_ni[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s];
    for (int kk = l; kk < ng; kk += 32) {
        const int pt = p.slot_partner[so + kk];
        const int gi = p.slot_g[so + kk];
        const double z = __ldcg(p.zl + so + kk) + (pt >= 0 ? __ldcg(p.zl + pt) : 0.0);
        const double dn = (k == 0) ? z : z + beta * __ldcg(dold + gi);
        if (slot_owner((int)(so + kk), pt)) dnew[gi] = dn;
        w.x[kk] = dn;
    }
    const double dpn = (k == 0) ? __ldcg(p.zp + s) : __ldcg(p.zp + s) + beta * __ldcg(dpold + s);
    if (l == 0) dpnew[s] = dpn;
    __syncwarp();
    // extension: column j of G_post (input-major) holds the outputs of
    // interface input j, interior fluxes then cell pressures; staged in the
    // warp's area after tsum (max_ext doubles)
    double* ext = w.tsum + p.max_m + 1;
    const double* G = p.Gpost + p.off_Gpost[s];
    const int no = ni + nc;
    for (int o = l; o < no; o += 32) {
        double a0 = 0.0, a1 = 0.0;
        int j = 0;
        for (; j + 1 < ng; j += 2) {
            a0 = fma(__ldg(G + (int64_t)j * no + o), w.x[j], a0);
            a1 = fma(__ldg(G + (int64_t)(j + 1) * no + o), w.x[j + 1], a1);
        }
        if (j < ng) a0 = fma(__ldg(G + (int64_t)j * no + o), w.x[j], a0);
        ext[o] = a0 + a1;
    }
    __syncwarp();
    constexpr double kThird = 1.0 / 3.0, kSixth = 1.0 / 6.0;
    const double ds = p.sub_d[s];
    double dq = 0.0;
    for (int kk = l; kk < ng; kk += 32) {
        const int op = p.slot_fopp[so + kk], pc = p.slot_fcell[so + kk];
        const double ue = w.x[kk];
        const double uo = op < 0 ? 0.0 : (op < ng ? w.x[op] : ext[op - ng]);
        const double pk = ds * (dpn + ext[ni + (pc > 0 ? pc : -pc) - 1]);
        const double q = p.slot_fk[so + kk] * (kThird * ue + kSixth * uo) + (pc > 0 ? pk : -pk);
        p.ql[so + kk] = q;
        dq += ue * q;
    }
    dq = warp_sum(dq);
    if (l == 0) p.part_dq[u] = dq;  // one unit per subdomain in the full form
    __syncwarp();
    return true;
}

template <class PR>
__device__ bool ph_update(const Params& p, int64_t s, int k, WarpSm w) {
    const int b = p.sub_inst[s];
    if (inst_done(p, b)) return false;
    const int l = threadIdx.x & 31;
    const double alpha = __ldcg(p.alpha_hist + (int64_t)b * (p.maxit + 1) + k);
    const double* rold = (k & 1) ? p.rbuf1 : p.rbuf0;
    double* rnew = (k & 1) ? p.rbuf0 : p.rbuf1;
    const double* dcur = (k & 1) ? p.dbuf1 : p.dbuf0;
    const double* dpcur = (k & 1) ? p.dp1 : p.dp0;
    const int ng = p.sub_ng[s];
    const int64_t so = p.off_slot[s];
    double rr = 0.0;
    for (int kk = l; kk < ng; kk += 32) {
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
        w.x[kk] = wr;
        p.rl[so + kk] = wr;
    }
    rr = warp_sum(rr);
    if (l == 0) {
        p.part_rr[s] = rr;
        p.xp[s] = __ldcg(p.xp + s) + alpha * __ldcg(dpcur + s);
    }
    __syncwarp();
    restrict_apply<PR>(p, s, w);
    return true;
}

// mixed path: FP64 restriction of the final residual for the closing coarse
// pressure correction
__device__ void ph_final_restrict(const Params& p, int64_t s, WarpSm w) {
    const int b = p.sub_inst[s];
    const int ng = p.sub_ng[s], m = p.sub_m[s];
    const int64_t so = p.off_slot[s], co = p.off_cslot[s];
    const int it = __ldcg(&p.st[b].iterations);
    const double* r = (it & 1) ? p.rbuf1 : p.rbuf0;
    for (int k = threadIdx.x & 31; k < ng; k += 32) w.x[k] = p.slot_w[so + k] * __ldcg(r + p.slot_g[so + k]);
    __syncwarp();
    restrict_rows(p.P64 + p.off_P[s], m, ng, w, p.rcl + co);
    __syncwarp();
}

__device__ void ph_final_pressure(const Params& p, int64_t s) {
    if ((threadIdx.x & 31) != 0) return;
    const int b = p.sub_inst[s];
    const double* wcb = p.wc + p.inst_coff[b];
    p.xp[s] = __ldcg(p.xp + s) + __ldcg(wcb + p.inst_ncf[b] + p.sub_local[s]);
}

__device__ void ph_post(const Params& p, int64_t s, WarpSm w) {
    const int ng = p.sub_ng[s], ni = p.sub_ni[s], nc = p.sub_nc[s];
    const int64_t so = p.off_slot[s], cb = p.off_cell[s], ib = p.off_int[s];
    const int l = threadIdx.x & 31;
    for (int k = l; k < ng; k += 32) {
        const int gi = p.slot_g[so + k];
        const double u = __ldcg(p.u0 + gi) + __ldcg(p.x + gi);
        if (slot_owner((int)(so + k), p.slot_partner[so + k])) p.flux_out[p.g_fid[gi]] = u;
        w.xin[k] = u;
    }
    int nz = 0;
    for (int r = l; r < nc; r += 32) {
        const double fv = p.f_in[p.cell_gid[cb + r]];
        w.xin[ng + r] = fv;
        nz |= (fv != 0.0);
    }
    // a subdomain without sources has f = 0: its f columns contribute exactly nothing
    const int nin = ng + (__any_sync(0xffffffffu, nz) ? nc : 0);
    __syncwarp();
    const double* G = p.Gpost + p.off_Gpost[s];
    const int no = ni + nc;
    const double d = p.sub_d[s];
    const double xp = __ldcg(p.xp + s);
    for (int o = l; o < no; o += 32) {
        double a0 = 0.0, a1 = 0.0;
        int j = 0;
        for (; j + 1 < nin; j += 2) {
            a0 = fma(__ldg(G + (int64_t)j * no + o), w.xin[j], a0);
            a1 = fma(__ldg(G + (int64_t)(j + 1) * no + o), w.xin[j + 1], a1);
        }
        if (j < nin) a0 = fma(__ldg(G + (int64_t)j * no + o), w.xin[j], a0);
        const double v = a0 + a1;
        if (o < ni) p.flux_out[p.int_fid[ib + o]] = v;
        else p.p_out[p.cell_gid[cb + o - ni]] = d * (xp + v);
    }
    __syncwarp();
}

#include "bddc_mixed.cuh"

// ---- sparse coarse solver: sweeps over the multifrontal factor ------------------------
// (bddc_coarse.cpp builds the factor; this is its solve, FP64 on both paths)
//
// right-hand sides of every instance's coarse system (grid-stride over all
// entries; a coarse problem has up to ~1e5 dofs): the flux part sums the
// two coarse slots of each coarse flux dof, the pressure part is the Step-1
// right-hand side (step1) or zero; the pure-flux multiplier row is zero
template <class PR>
__device__ void cs_rhs(const Params& p, bool step1) {
    const int64_t total = p.inst_csoff[p.n_inst];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = p.n_inst - 1;  // the instance: last b with inst_csoff[b] <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.inst_csoff[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const int b = lo;
        const int64_t ncf = p.inst_ncf[b], ncn = p.inst_ncn[b], cfo = p.inst_cfoff[b], s0 = p.inst_s0[b];
        const int64_t cs = p.inst_csoff[b], c = g - cs;
        double v = 0.0;
        if (c < ncf) {
            const int a = p.c_slot_a[cfo + c], bb = p.c_slot_b[cfo + c];
            if constexpr (PR::kMixed) {
                const float2* rcl = reinterpret_cast<const float2*>(p.rcl);
                v = (a >= 0 ? dd_dbl(__ldcg(rcl + a)) : 0.0) + (bb >= 0 ? dd_dbl(__ldcg(rcl + bb)) : 0.0);
            } else {
                v = (a >= 0 ? __ldcg(p.rcl + a) : 0.0) + (bb >= 0 ? __ldcg(p.rcl + bb) : 0.0);
            }
        } else if (c < ncn && step1) {
            v = __ldcg(p.prhs + s0 + (c - ncf));
        }
        p.cs_b[g] = v;
    }
}

// Both sweeps are GEMVs with the node's dense blocks; their dot products are
// split into chunks of kCsChunk terms so that a level's work spreads over
// many warps (the top fronts have ~1000 columns).  Each unit (node, block
// of 32 outputs, chunk) stores its partial sums; the unit whose arrival
// completes a block sums the partials in chunk order (independent of the
// arrival order) and writes the block.  A block with one chunk writes
// directly.  The chunk is fixed per node (not per batch), so an instance
// gets the same bits alone and in a batch.
//
// A unit is latency-bound (a level has about one unit per warp), so it is
// laid out for few dependent round trips: its record (CsUnit) in one load
// batch; then the first half of its matrix chunk, the front indices and the
// completion's indices together; then the right-hand-side values and the
// children's updates together; then the second half of the matrix chunk.

// the last of n arrivals at *cnt (whole warp; the completing warp resets it)
__device__ __forceinline__ bool cs_arrive_last(int* cnt, int n) {
    int last = 0;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        last = arrive_acq_rel(cnt) == n - 1;
        if (last) *cnt = 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) __threadfence();
    return last != 0;
}

__device__ __forceinline__ CsUnit cs_load_unit(const CsUnit* u) {
    CsUnit U;
    const int4* src = reinterpret_cast<const int4*>(u);
    int4* dst = reinterpret_cast<int4*>(&U);
#pragma unroll
    for (int t = 0; t < (int)(sizeof(CsUnit) / sizeof(int4)); ++t) dst[t] = __ldg(src + t);
    return U;
}

// acc += sum_{k < kh} m[k] * (value of column k, held by lane k of the warp)
template <int kh>
__device__ __forceinline__ double cs_dot(const double (&m)[kh], double v, int lane0, double acc) {
    // lane0 + kh <= 32: the chunk has at most 32 terms, one per lane
#pragma unroll
    for (int k = 0; k < kh; ++k) acc = fma(m[k], __shfl_sync(0xffffffffu, v, lane0 + k), acc);
    return acc;
}

// forward unit (node v, block of 32 boundary rows j, chunk of its pivots):
// t_i = b_i + the children's updates for the chunk's pivots (stored for the
// backward sweep by the units of block 0), partial (H^T t)_j over the
// chunk; the block's u_j = children's updates - the sum of the partials
__device__ void cs_forward(const Params& p, const CsUnit& U) {
    constexpr int kh = 8;  // matrix entries in flight per lane
    const int l = threadIdx.x & 31;
    const int j = U.blk * 32 + l;
    const int nk = U.k1 - U.k0;
    const bool jin = j < U.q;
    const double* Hc = p.cn_H + (int64_t)U.om + (int64_t)U.k0 * U.q + j;
    if (l < nk && U.q > U.blk * 32)
        prefetch_l2_row32(p.cn_H + (int64_t)U.om + (int64_t)(U.k0 + l) * U.q + U.blk * 32, min(32, U.q - U.blk * 32));
    double m[kh];
#pragma unroll
    for (int k = 0; k < kh; ++k) m[k] = (k < nk && jin) ? __ldg(Hc + (int64_t)k * U.q) : 0.0;
    int4 ix = make_int4(-1, -1, -1, 0), jx = make_int4(-1, -1, -1, 0);
    if (l < nk) ix = __ldg(p.cn_idx + (int64_t)U.od + U.k0 + l);
    if (jin) jx = __ldg(p.cn_idx + (int64_t)U.od + U.pp + j);
    double tl = 0.0, ch = 0.0;
    if (l < nk) {
        tl = __ldcg(p.cs_b + U.cs + ix.x) + (ix.y >= 0 ? __ldcg(p.cs_u + ix.y) : 0.0) +
             (ix.z >= 0 ? __ldcg(p.cs_u + ix.z) : 0.0);
        if (U.blk == 0) p.cs_t[U.cs + ix.x] = tl;
    }
    if (jin) ch = (jx.y >= 0 ? __ldcg(p.cs_u + jx.y) : 0.0) + (jx.z >= 0 ? __ldcg(p.cs_u + jx.z) : 0.0);
    double acc = cs_dot(m, tl, 0, 0.0);
    for (int k0 = kh; k0 < nk; k0 += kh) {
#pragma unroll
        for (int k = 0; k < kh; ++k) m[k] = (k0 + k < nk && jin) ? __ldg(Hc + (int64_t)(k0 + k) * U.q) : 0.0;
        acc = cs_dot(m, tl, k0, acc);
    }
    if (U.q == 0) return;  // the root: only its t
    if (U.nch > 1) {
        double* part = p.cs_fpart + U.pof;
        part[(int64_t)U.ich * 32 + l] = acc;
        if (!cs_arrive_last(p.cs_fcnt + U.cof, U.nch)) return;
        acc = 0.0;
        for (int c = 0; c < U.nch; ++c) acc += __ldcg(part + (int64_t)c * 32 + l);
    }
    if (jin) p.cs_u[U.ou + j] = ch - acc;
}

// backward unit (node v, block of 32 pivot rows i, chunk of the
// concatenated columns [P, B]): partial of x_i = sum_k X_ik t_k -
// sum_j H_ij x_j (X symmetric: X_ik read as X[k][i]; H from its transpose);
// the completed block goes to cs_x and, for the n_c + N coarse dofs, to wc
template <class PR>
__device__ void cs_backward(const Params& p, const CsUnit& U) {
    constexpr int kh = 8;  // matrix entries in flight per lane
    const int l = threadIdx.x & 31;
    const int i = U.blk * 32 + l;
    const int nk = U.k1 - U.k0;
    const bool iin = i < U.pp;
    // column k of the chunk is kk = k0 + k: X row kk (kk < p), else -H^T row kk - p
    auto mat = [&](int k) -> double {
        const int kk = U.k0 + k;
        if (k >= nk || !iin) return 0.0;
        return kk < U.pp ? __ldg(p.cn_X + (int64_t)U.om + (int64_t)kk * U.pp + i)
                         : -__ldg(p.cn_HT + (int64_t)U.ou + (int64_t)(kk - U.pp) * U.pp + i);
    };
    if (l < nk && U.pp > U.blk * 32) {
        const int kk = U.k0 + l;
        prefetch_l2_row32(kk < U.pp ? p.cn_X + (int64_t)U.om + (int64_t)kk * U.pp + U.blk * 32
                                    : p.cn_HT + (int64_t)U.ou + (int64_t)(kk - U.pp) * U.pp + U.blk * 32,
                          min(32, U.pp - U.blk * 32));
    }
    double m[kh];
#pragma unroll
    for (int k = 0; k < kh; ++k) m[k] = mat(k);
    int dl = -1, di = -1;
    if (l < nk) dl = __ldg(p.cn_idx + (int64_t)U.od + U.k0 + l).x;
    if (iin) di = __ldg(p.cn_idx + (int64_t)U.od + i).x;
    // the column values: t at pivots, x at boundary dofs (set one level up)
    double vl = 0.0;
    if (l < nk) vl = __ldcg((U.k0 + l < U.pp ? p.cs_t : p.cs_x) + U.cs + dl);
    double acc = cs_dot(m, vl, 0, 0.0);
    for (int k0 = kh; k0 < nk; k0 += kh) {
#pragma unroll
        for (int k = 0; k < kh; ++k) m[k] = mat(k0 + k);
        acc = cs_dot(m, vl, k0, acc);
    }
    if (U.nch > 1) {
        double* part = p.cs_bpart + U.pof;
        part[(int64_t)U.ich * 32 + l] = acc;
        if (!cs_arrive_last(p.cs_bcnt + U.cof, U.nch)) return;
        acc = 0.0;
        for (int c = 0; c < U.nch; ++c) acc += __ldcg(part + (int64_t)c * 32 + l);
    }
    if (iin) {
        p.cs_x[U.cs + di] = acc;
        if (di < p.inst_ncn[U.b]) {
            if constexpr (PR::kMixed) reinterpret_cast<float2*>(p.wc)[p.inst_coff[U.b] + di] = dd_of(acc);
            else p.wc[p.inst_coff[U.b] + di] = acc;
        }
    }
}

// ---- the persistent solve kernel -------------------------------------------------------
// kBal: the CG phases of a batch are rebalanced over the instances still
// active (g_partial_sh, active_snapshot); without it (one instance, or more
// than kActMaxInst) every phase keeps its work-balanced static ranges.  Two
// instantiations, because the kernel runs at its register cap and the
// rebalancing's bookkeeping changes the register allocation of the phases.
template <class PR, bool kBal>
__global__ void __launch_bounds__(kThreads, 4) bddc_solve_kernel(Params p) {
    constexpr bool MX = PR::kMixed;
    extern __shared__ double smem_base[];
    // the shared-memory areas are formed where a unit uses them, so that no
    // register holds their addresses across the phases (the kernel runs at
    // its register cap); the CTA's coarse right-hand side starts the area
    auto wsm = [&]() { return carve<PR::kFull>(p, smem_base).w; };
    int64_t a, e;
    int staged;
    int nts = 0;
    // sparse coarse solve: the first unit of every depth, forward then backward
    __shared__ int64_t cs_lvl[2 * (kCsMaxLevels + 1)];
    if (p.coarse_sparse && p.cn_levels <= kCsMaxLevels)
        for (int d = threadIdx.x; d <= p.cn_levels; d += kThreads) {
            cs_lvl[d] = p.fw_off[d];
            cs_lvl[kCsMaxLevels + 1 + d] = p.bw_off[d];
        }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.tstamp && p.tstamp_cap > 0) {
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        p.tstamp[0] = 0;
        p.tstamp[1] = t;
        nts = 1;
    }
    // g_partial_sh (per CG iteration): some instances have left the loop,
    // and the CG phases spread the active instances' work over all warps
    // and CTAs
    if (threadIdx.x == 0) g_partial_sh = 0;
    auto coarse_phase = [&](bool step1) {
        staged = -1;
        // with g_partial_sh the active instances' coarse units are split
        // evenly over the CTAs (unit position x -> the x-th active unit)
        const bool part = kBal && !step1 && g_partial_sh;
        if (part) {
            const int* act_cu = act_area<PR::kFull>(p, smem_base) + p.act_n + 1;
            cta_range(act_cu[p.act_n], a, e);
        } else {
            cta_range(p.n_cunits, a, e);
        }
        for (int64_t x = a; x < e; ++x) {
            int64_t u = x;
            if (part) {
                const int* act_cu = act_area<PR::kFull>(p, smem_base) + p.act_n + 1;
                const int b = act_find(act_cu, p.act_n, x);
                u = p.inst_cu0[b] + (x - act_cu[b]);
            }
            if constexpr (MX) mx_coarse(p, u, step1, smem_base, staged);
            else ph_coarse<PR>(p, u, step1, smem_base, staged);
        }
    };
    // a coarse solve and the grid barrier(s) after it: the dense inverse in
    // one phase, or the sparse factor's right-hand side, forward sweep (tree
    // depths deepest first) and backward sweep (root first), a phase each.
    // Between the CG iterations, instances that are done skip their units.
    auto coarse_solve = [&](bool step1, int id) -> bool {
        if (!p.coarse_sparse) {
            coarse_phase(step1);
            return phase_end(p, id, nts);
        }
        cs_rhs<PR>(p, step1);
        if (!phase_end(p, id, nts)) return false;
        // the unit offsets per depth: from shared memory (staged at the start)
        // when the tree is not deeper than kCsMaxLevels
        const bool lvl_sh = p.cn_levels <= kCsMaxLevels;
        for (int d = p.cn_levels - 1; d >= 0; --d) {
            const int64_t u0 = lvl_sh ? cs_lvl[d] : p.fw_off[d];
            warp_range((lvl_sh ? cs_lvl[d + 1] : p.fw_off[d + 1]) - u0, a, e);
            for (int64_t u = a; u < e; ++u) {
                const CsUnit U = cs_load_unit(p.fw_unit + u0 + u);
                if (step1 || p.n_inst == 1 || !inst_done(p, U.b)) cs_forward(p, U);
            }
            if (!phase_end(p, id, nts)) return false;
        }
        for (int d = 0; d < p.cn_levels; ++d) {
            const int64_t u0 = lvl_sh ? cs_lvl[kCsMaxLevels + 1 + d] : p.bw_off[d];
            warp_range((lvl_sh ? cs_lvl[kCsMaxLevels + 2 + d] : p.bw_off[d + 1]) - u0, a, e);
            for (int64_t u = a; u < e; ++u) {
                const CsUnit U = cs_load_unit(p.bw_unit + u0 + u);
                if (step1 || p.n_inst == 1 || !inst_done(p, U.b)) cs_backward<PR>(p, U);
            }
            if (!phase_end(p, id, nts)) return false;
        }
        return true;
    };
    sub_range(p, a, e);
    for (int64_t s = a; s < e; ++s) {
        if constexpr (MX) mx_step1(p, s, wsm());
        else ph_step1<PR>(p, s, wsm());
    }
    if (!phase_end(p, 1, nts)) return;
    if (!coarse_solve(true, 2)) return;
    sub_range(p, a, e);
    for (int64_t s = a; s < e; ++s) {
        if constexpr (MX) mx_u0(p, s, wsm());
        else ph_u0<PR>(p, s, wsm());
    }
    if (!phase_end(p, 3, nts)) return;
    for (int64_t s = a; s < e; ++s) ph_step2<PR>(p, s, wsm());
    if (!phase_end(p, 4, nts)) return;
    for (int64_t s = a; s < e; ++s) {
        if constexpr (MX) mx_fstar(p, s, wsm());
        else ph_fstar<PR>(p, s, wsm());
    }
    if (!phase_end(p, 5, nts)) return;
    if (!coarse_solve(false, 6)) return;
    // a CG phase over the warp's subdomains; the arrivals of its consecutive
    // subdomains of one instance are counted at once (publish_total)
    auto cg_phase = [&](int ctr, int kk, auto&& unit) {
        // positions [a, e) of this warp: its work-balanced subdomain range,
        // or with g_partial_sh an even share of the active instances'
        // subdomains in instance order (by count: the subdomains of a batch
        // are alike), position x -> the x-th active subdomain
        if (kBal && g_partial_sh) {
            const int64_t A = act_area<PR::kFull>(p, smem_base)[p.act_n];
            const int64_t W = (int64_t)gridDim.x * kWarps;
            const int64_t wg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
            a = (A * wg) / W;
            e = (A * (wg + 1)) / W;
        } else {
            sub_range(p, a, e);
        }
        int cur = -1, n = 0;
        for (int64_t x = a; x < e; ++x) {
            int64_t s = x;
            int b;
            if (kBal && g_partial_sh) {
                const int* act_sub = act_area<PR::kFull>(p, smem_base);
                b = act_find(act_sub, p.act_n, x);
                s = p.inst_s0[b] + (x - act_sub[b]);
            } else {
                b = p.sub_inst[s];
            }
            if (b != cur) {
                if (n > 0) publish_total(p, cur, n, ctr, kk, false, !MX);
                cur = b;
                n = 0;
            }
            if (unit(s)) ++n;
        }
        if (n > 0) publish_total(p, cur, n, ctr, kk, false, !MX);
    };
    // each PROLONG ends with the convergence test of the next iteration
    auto prolong_unit = [&](int64_t s) -> bool {
        if constexpr (MX) return mx_prolong(p, s, wsm());
        else return ph_prolong<PR>(p, s, wsm());
    };
    cg_phase(kCtrRZ, 0, prolong_unit);
    if (!phase_end(p, 7, nts)) return;
    for (int k = 0;; ++k) {
        // the instances still in the loop: every CTA takes the same snapshot
        // (phase_index), so all leave the loop at the same iteration; with
        // more than kActMaxInst instances the count of active instances is
        // read instead (the snapshot is off)
        if (p.act_n > 0) {
            if (active_snapshot(p, act_area<PR::kFull>(p, smem_base), phase_index(k, kPhDirop)) == 0) break;
        } else if (__ldcg(p.n_active) <= 0) {
            break;
        }
        // DIROP over the operator-apply units: the warp's work-balanced unit
        // range, or with g_partial_sh the units of its even share of the
        // active instances' subdomains
        {
            int cur = -1, n = 0;
            auto dirop_unit = [&](int64_t u) {
                const int2 du = __ldg(p.dunit + u);
                const int b = p.sub_inst[du.x];
                if (b != cur) {
                    if (n > 0) publish_total(p, cur, n, kCtrDQ, k, false, !MX);
                    cur = b;
                    n = 0;
                }
                bool ok;
                if constexpr (MX) ok = mx_dirop(p, u, du.x, du.y >> 16, du.y & 0xffff, k, wsm());
                else if constexpr (PR::kFull) ok = ph_dirop_full<PR>(p, u, du.x, k, wsm());
                else ok = ph_dirop<PR>(p, u, du.x, du.y >> 16, du.y & 0xffff, k, wsm());
                if (ok) ++n;
            };
            if (kBal && g_partial_sh) {
                const int64_t A = act_area<PR::kFull>(p, smem_base)[p.act_n];
                const int64_t W = (int64_t)gridDim.x * kWarps;
                const int64_t wg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
                a = (A * wg) / W;
                e = (A * (wg + 1)) / W;
                for (int64_t x = a; x < e; ++x) {
                    const int* act_sub = act_area<PR::kFull>(p, smem_base);
                    const int b = act_find(act_sub, p.act_n, x);
                    const int64_t sx = p.inst_s0[b] + (x - act_sub[b]);
                    for (int64_t u = p.sub_du0[sx]; u < p.sub_du0[sx + 1]; ++u) dirop_unit(u);
                }
            } else {
                const int64_t wg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
                a = p.warp_du0[wg];
                e = p.warp_du0[wg + 1];
                for (int64_t u = a; u < e; ++u) dirop_unit(u);
            }
            if (n > 0) publish_total(p, cur, n, kCtrDQ, k, false, !MX);
        }
        if (!phase_end(p, 8, nts)) return;
        cg_phase(kCtrRR, k, [&](int64_t s) -> bool {
            if constexpr (MX) return mx_update(p, s, k, wsm());
            else return ph_update<PR>(p, s, k, wsm());
        });
        if (!phase_end(p, 9, nts)) return;
        if (!coarse_solve(false, 6)) return;
        cg_phase(kCtrRZ, k + 1, prolong_unit);
        if (!phase_end(p, 7, nts)) return;
    }
    __syncthreads();
    if (threadIdx.x == 0) g_partial_sh = 0;
    __syncthreads();
    if constexpr (MX) {
        // closing FP64 coarse pressure correction (every instance is done;
        // the coarse phase runs in step-1 layout with a zero pressure part)
        sub_range(p, a, e);
        for (int64_t s = a; s < e; ++s) mx_final_restrict(p, s, wsm());
        if (!phase_end(p, 10, nts)) return;
        cta_range(p.n_sub, a, e);
        for (int64_t s = a; s < e; ++s)
            if (threadIdx.x == 0) p.prhs[s] = 0.0;
        if (!phase_end(p, 11, nts)) return;
        if (!coarse_solve(true, 12)) return;
        sub_range(p, a, e);
        for (int64_t s = a; s < e; ++s) mx_final_pressure(p, s);
        if (!phase_end(p, 13, nts)) return;
    }
    sub_range(p, a, e);
    for (int64_t s = a; s < e; ++s) {
        if constexpr (MX) mx_post(p, s, wsm());
        else ph_post(p, s, wsm());
    }
}

// ---- stand-alone operator / preconditioner kernels (grid-stride over units) --------
template <class PR>
__global__ void __launch_bounds__(kThreads) k_operator_local(Params p, const double* u, const double* p0) {
    using S_t = typename PR::S_t;
    extern __shared__ double smem_base[];
    CtaSm sm = carve(p, smem_base);
    WarpSm& w = sm.w;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < p.n_sub; s += W) {
        const int ng = p.sub_ng[s];
        const int64_t so = p.off_slot[s];
        for (int k = threadIdx.x & 31; k < ng; k += 32) w.x[k] = u[p.slot_g[so + k]];
        __syncwarp();
        if constexpr (PR::kMixed) split_pairs(w, ng);
        const S_t* S = reinterpret_cast<const S_t*>(p.S) + p.off_S[s];
        const double pv = p0[s];
        gemv_warp(S, ng, w, [&](int k, typename GAcc<S_t>::value_type y) {
            p.ql[so + k] = to_double(y) + p.slot_dsig[so + k] * pv;
        });
        __syncwarp();
    }
}

__global__ void k_assemble(int64_t n_slots, const double* loc, const int* slot_g, const int* partner, double* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_slots; q += (int64_t)gridDim.x * blockDim.x) {
        const int pt = partner[q];
        if (pt >= 0 && pt < q) continue;
        out[slot_g[q]] = loc[q] + (pt >= 0 ? loc[pt] : 0.0);
    }
}

template <class PR>
__global__ void __launch_bounds__(kThreads) k_precond_restrict(Params p, const double* r) {
    extern __shared__ double smem_base[];
    CtaSm sm = carve(p, smem_base);
    WarpSm& w = sm.w;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < p.n_sub; s += W) {
        const int ng = p.sub_ng[s];
        const int64_t so = p.off_slot[s];
        for (int k = threadIdx.x & 31; k < ng; k += 32) {
            const double wr = p.slot_w[so + k] * r[p.slot_g[so + k]];
            w.x[k] = wr;
            p.rl[so + k] = wr;
        }
        __syncwarp();
        restrict_apply<PR>(p, s, w);
    }
}

template <class PR>
__global__ void __launch_bounds__(kThreads) k_precond_coarse(Params p) {
    extern __shared__ double smem_base[];
    CtaSm sm = carve(p, smem_base);
    for (int64_t u = blockIdx.x; u < p.n_cunits; u += gridDim.x) {
        int staged = -1;
        ph_coarse<PR>(p, u, false, sm.rhs, staged);
    }
}

// sparse coarse solve of the stand-alone preconditioner: right-hand sides,
// then one launch per tree depth and sweep
template <class PR>
__global__ void __launch_bounds__(kThreads) k_cs_rhs(Params p) {
    cs_rhs<PR>(p, false);
}
__global__ void __launch_bounds__(kThreads) k_cs_forward(Params p, int d) {
    const int64_t W = (int64_t)gridDim.x * kWarps, u0 = p.fw_off[d], nu = p.fw_off[d + 1] - u0;
    for (int64_t u = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); u < nu; u += W) {
        cs_forward(p, cs_load_unit(p.fw_unit + u0 + u));
    }
}
template <class PR>
__global__ void __launch_bounds__(kThreads) k_cs_backward(Params p, int d) {
    const int64_t W = (int64_t)gridDim.x * kWarps, u0 = p.bw_off[d], nu = p.bw_off[d + 1] - u0;
    for (int64_t u = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); u < nu; u += W) {
        cs_backward<PR>(p, cs_load_unit(p.bw_unit + u0 + u));
    }
}

template <class PR>
__global__ void __launch_bounds__(kThreads) k_precond_prolong(Params p, double* z0) {
    using F_t = typename PR::F_t;
    extern __shared__ double smem_base[];
    CtaSm sm = carve(p, smem_base);
    WarpSm& w = sm.w;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < p.n_sub; s += W) {
        const int b = p.sub_inst[s];
        const int ng = p.sub_ng[s], m = p.sub_m[s];
        const int64_t so = p.off_slot[s];
        const double* wcb = p.wc + p.inst_coff[b];
        stage_wc(p, s, wcb, w);
        const F_t* P = reinterpret_cast<const F_t*>(p.P) + p.off_P[s];
        for (int k = threadIdx.x & 31; k < ng; k += 32) w.xin[k] = prolong_out(P, m, ng, w, k);
        __syncwarp();
        if constexpr (PR::kMixed) {
            face_sums(p, s, w.xin, w.tsum);
            set_face_flux(p, s, w.xin, w.tsum, w.wcs);
        }
        for (int k = threadIdx.x & 31; k < ng; k += 32) p.zl[so + k] = p.slot_w[so + k] * (w.xin[k] + p.yl[so + k]);
        if ((threadIdx.x & 31) == 0) z0[s] = wcb[p.inst_ncf[b] + p.sub_local[s]];
        __syncwarp();
    }
}

// ---- true residual of the full saddle system (matrix-free RT0/P0) -----------------
// For the solution (u, p) of instance b, the residuals of both block rows of
// the discrete system of Sec. 2 (eqs. (a), (b), (rhs); the pressure faces
// carry g = +-p_N on the min / max side): on every free face e
//   r_e = g_e - sum over its two cells c of (a_c u)_e - (B^T p)_e,
// with the exact RT0 cell block (h_a^2 / |c|) k_a^-1 [1/3 1/6; 1/6 1/3] on
// the two a-faces of a cell and B(c, lower face) = +1, B(c, upper face) = -1;
// on every cell  r_c = -f_c |c| - (B u)_c.  CTA (b, chunk) covers a chunk of
// instance b's faces and cells and writes its sums of r_e^2, g_e^2, r_c^2
// and (f_c |c|)^2; k_true_residual_sum adds the chunks in order (a fixed
// summation order: bitwise reproducible) and writes
// sqrt(sum r^2) / sqrt(sum rhs^2) per instance.
constexpr int kTrChunks = 16;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) t += sh[w];
    return t;  // valid on thread 0
}

__global__ void __launch_bounds__(kThreads) k_true_residual(Params p) {
    __shared__ double sh[kWarps];
    const int b = blockIdx.x / kTrChunks, chunk = blockIdx.x % kTrChunks;
    // 32-bit index arithmetic: an instance has < 2^31 faces
    const int dim = p.inst_grid[4 * b], nx = p.inst_grid[4 * b + 1], ny = p.inst_grid[4 * b + 2],
              nz = p.inst_grid[4 * b + 3];
    const double* h = p.inst_h + 3 * b;
    const double vol = h[0] * h[1] * (dim == 3 ? h[2] : 1.0);
    const int64_t f0 = p.inst_face_off[b], c0 = p.inst_cell_off[b];
    const double* u = p.flux_out + f0;
    const double* pr = p.p_out + c0;
    const int8_t* bct = p.face_bct + f0;
    const double* bcv = p.bc_in + f0;
    const double* kinv = p.cell_kinv + 3 * c0;
    double r1 = 0.0, g2 = 0.0, r2 = 0.0, f2 = 0.0;
    int off = 0;  // first face of axis a
    for (int a = 0; a < dim; ++a) {
        const unsigned ex = nx + (a == 0), ey = ny + (a == 1), ez = nz + (a == 2 && dim == 3);
        const unsigned cnt = ex * ey * ez;
        const unsigned na = a == 0 ? nx : (a == 1 ? ny : nz);
        const unsigned step = a == 0 ? 1u : (a == 1 ? ex : ex * ey);                    // face id step along a
        const unsigned cstep = a == 0 ? 1u : (a == 1 ? (unsigned)nx : (unsigned)nx * ny);  // cell id step along a
        const double s = h[a] * h[a] / vol;
        const unsigned fa = (unsigned)((uint64_t)cnt * chunk / kTrChunks), fb = (unsigned)((uint64_t)cnt * (chunk + 1) / kTrChunks);
        for (unsigned r = fa + threadIdx.x; r < fb; r += kThreads) {
            const int e = off + (int)r;
            const int bt = bct[e];
            if (bt == 0) continue;  // no-flow face: not an unknown
            const unsigned i = r % ex, jk = r / ex, j = jk % ey, k = jk / ey;
            const unsigned pos = a == 0 ? i : (a == 1 ? j : k);
            // the cell above the face along a has the face's indices; the one below is a step back
            const unsigned ci = i + (unsigned)nx * (j + (unsigned)ny * k);
            const double ue = u[e];
            double au = 0.0, btp = 0.0;
            // the RT0 cell block entries 1/3 and 1/6 as products: FP64 division
            // is a long instruction sequence at GB300's FP64 rate
            constexpr double kThird = 1.0 / 3.0, kSixth = 1.0 / 6.0;
            if (pos < na) {  // e is the lower a-face of the cell above
                au += s * kinv[3 * ci + a] * (kThird * ue + kSixth * u[e + step]);
                btp += pr[ci];
            }
            if (pos > 0) {  // e is the upper a-face of the cell below
                const unsigned c = ci - cstep;
                au += s * kinv[3 * c + a] * (kSixth * u[e - step] + kThird * ue);
                btp -= pr[c];
            }
            const double g = bt == 1 ? (pos == 0 ? bcv[e] : -bcv[e]) : 0.0;
            const double res = g - au - btp;
            r1 += res * res;
            g2 += g * g;
        }
        off += (int)cnt;
    }
    // cells: per axis the lower face is at (i, j, k) of the axis' face grid
    const unsigned ncell = (unsigned)nx * ny * nz;
    const unsigned ca = (unsigned)((uint64_t)ncell * chunk / kTrChunks), cb = (unsigned)((uint64_t)ncell * (chunk + 1) / kTrChunks);
    const unsigned fo1 = (unsigned)(nx + 1) * ny * nz, fo2 = fo1 + (unsigned)nx * (ny + 1) * nz;
    for (unsigned c = ca + threadIdx.x; c < cb; c += kThreads) {
        const unsigned i = c % nx, jk = c / nx, j = jk % ny, k = jk / ny;
        const unsigned lx = i + (nx + 1) * (j + (unsigned)ny * k);
        const unsigned ly = fo1 + i + (unsigned)nx * (j + (unsigned)(ny + 1) * k);
        double div = (u[lx] - u[lx + 1]) + (u[ly] - u[ly + nx]);
        if (dim == 3) {
            const unsigned lz = fo2 + i + (unsigned)nx * (j + (unsigned)ny * k);
            div += u[lz] - u[lz + (unsigned)nx * ny];
        }
        const double rhs = -p.f_in[c0 + c] * vol;
        const double res = rhs - div;
        r2 += res * res;
        f2 += rhs * rhs;
    }
    double* out = p.tr_part + 4 * (int64_t)blockIdx.x;
    const double s1 = block_sum(r1, sh);
    if (threadIdx.x == 0) out[0] = s1;
    const double s2 = block_sum(g2, sh);
    if (threadIdx.x == 0) out[1] = s2;
    const double s3 = block_sum(r2, sh);
    if (threadIdx.x == 0) out[2] = s3;
    const double s4 = block_sum(f2, sh);
    if (threadIdx.x == 0) out[3] = s4;
}

__global__ void k_true_residual_sum(Params p) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.n_inst) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < kTrChunks; ++c)
        for (int q = 0; q < 4; ++q) s[q] += p.tr_part[4 * ((int64_t)b * kTrChunks + c) + q];
    const double den = s[1] + s[3];
    p.tr_out[b] = sqrt(s[0] + s[2]) / (den > 0.0 ? sqrt(den) : 1.0);
}

// diagnostic of the bounded barrier wait: the last CTA never arrives, so
// the others give up after limit_ns and set the error flag
__global__ void k_barrier_probe(GridSync* gs, long long limit_ns) {
    if (blockIdx.x == gridDim.x - 1) return;
    grid_barrier(gs, limit_ns);
}

// FP64 -> FP32 pair (hi, lo) elementwise, on the device
__global__ void k_pairs(int64_t n, const double* src, float2* dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        const float hi = __double2float_rn(v);
        dst[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

// raw subassembled apply (no handle), from caller-owned index tables: the
// host has checked the sizes and the slot offsets; every index read from a
// caller table is also checked here against the buffer it addresses (slots
// against n_slots, interface indices against n_in), and an access outside
// is skipped, so bad table entries can give wrong values but never reach
// memory outside the caller's arrays and the scratch
__global__ void __launch_bounds__(128) k_subassembled_local(int n_sub, const int* ng_arr, const int64_t* slot_off,
                                                            const int64_t* S_off, const double* S, const int* gidx,
                                                            const double* u, double* scratch, int64_t n_slots,
                                                            int64_t n_in) {
    __shared__ double xs[1024];
    for (int s = blockIdx.x; s < n_sub; s += gridDim.x) {
        const int ng = ng_arr[s];
        const int64_t so = slot_off[s];
        for (int k = threadIdx.x; k < ng; k += blockDim.x) {
            const int64_t q = so + k;
            const int g = (q >= 0 && q < n_slots) ? gidx[q] : -1;
            xs[k] = (g >= 0 && g < n_in) ? u[g] : 0.0;
        }
        __syncthreads();
        const double* M = S + S_off[s];
        for (int k = threadIdx.x; k < ng; k += blockDim.x) {
            double acc = 0.0;
            for (int j = 0; j < ng; ++j) acc = fma(__ldg(M + (int64_t)j * ng + k), xs[j], acc);
            const int64_t q = so + k;
            if (q >= 0 && q < n_slots) scratch[q] = acc;
        }
        __syncthreads();
    }
}

// assembly of the raw apply: k_assemble with the partner slot and the
// output index checked against their buffers
__global__ void k_assemble_checked(int64_t n_slots, const double* loc, const int* slot_g, const int* partner,
                                   int64_t n_out, double* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_slots; q += (int64_t)gridDim.x * blockDim.x) {
        const int pt = partner[q];
        if (pt >= 0 && pt < q) continue;
        const int g = slot_g[q];
        if (g < 0 || g >= n_out || pt >= n_slots) continue;
        out[g] = loc[q] + (pt >= 0 ? loc[pt] : 0.0);
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
    int n_inst = 0, maxit = 0, precision = 0, formulation = BDDC_FORM_CONDENSED;
    Packed P;
    Params prm{};
    std::vector<void*> allocs;
    size_t dev_bytes = 0;  // device memory held by the handle
    std::string err;
    mutable std::vector<bddc_stats> stats;  // kappa filled on demand (bddc_get_stats)
    mutable bool kappa_stale = false;       // the last solve's kappa is not computed yet
    InstState* pin_st = nullptr;            // pinned read-back of the per-instance state
    double* pin_tr = nullptr;               // pinned read-back of the true residuals
    GridSync* pin_gs = nullptr;
    std::vector<int64_t> inst_cfoff;
    std::vector<int64_t> fw_off_h, bw_off_h;  // sparse coarse: units per tree depth (host copies)
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
    mutable std::vector<double> hist_a, hist_b;  // host copies of the CG coefficients
    bddc_tuning tuning{};                        // work layout of the solve launch
    std::vector<int2> dunit_h;                   // operator-apply units (host copy, for the warp ranges)
};

// message of the last failed setup of this thread (bddc_last_error(NULL));
// also set by the host-only setup in bddc_setup.cpp
thread_local std::string g_setup_err;

namespace {

const char* kErrStrings[] = {"ok", "invalid argument", "invalid partition", "invalid permeability",
                             "out of memory", "not converged", "CG breakdown", "device wait timed out",
                             "CUDA error", "setup factorisation failed"};


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
    h->dev_bytes += v.size() * sizeof(T);
    if (cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return BDDC_E_CUDA;
    *out = static_cast<const T*>(p);
    return BDDC_OK;
}

template <class T>
int dalloc(bddc_handle* h, size_t n, T** out) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return BDDC_E_OOM;
    h->allocs.push_back(p);
    h->dev_bytes += std::max<size_t>(n, 1) * sizeof(T);
    cudaMemset(p, 0, std::max<size_t>(n, 1) * sizeof(T));
    *out = static_cast<T*>(p);
    return BDDC_OK;
}

// Raise, never lower, a kernel's limit of dynamic shared memory.  The limit
// is one value per kernel for the whole process, and handles of different
// sizes are set up on several host threads (the serving loop) while earlier
// handles launch: lowering it for a small batch would make the launch of a
// larger one fail.
std::mutex g_smem_mu;
std::vector<std::pair<const void*, size_t>> g_smem_max;
bool ensure_smem(const void* fn, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    for (auto& e : g_smem_max)
        if (e.first == fn) {
            if (e.second >= bytes) return true;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
                return false;
            e.second = bytes;
            return true;
        }
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return false;
    g_smem_max.emplace_back(fn, bytes);
    return true;
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
    opt->coarse_solver = BDDC_COARSE_AUTO;
    opt->formulation = BDDC_FORM_CONDENSED;
    opt->constraints = BDDC_CONSTRAINTS_ADAPTIVE;
    opt->autotune = 0;
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
    if (h->pin_st) cudaFreeHost(h->pin_st);
    if (h->pin_tr) cudaFreeHost(h->pin_tr);
    if (h->pin_gs) cudaFreeHost(h->pin_gs);
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
    if (!bddc::options_valid(opt)) return BDDC_E_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return BDDC_E_CUDA;
    }
    Packed P;
    // dense local maps and face eigenproblems on the GPU
    SetupResult r = build_all(n_instances, inst, opt, P, local_maps_device, face_eigen_device);
    if (r.code) {
        g_setup_err = r.msg;
        return r.code;
    }
    return bddc::setup_from_packed(n_instances, opt, cuda_stream, std::move(P), out);
}

}  // extern "C"

namespace bddc {

size_t handle_device_bytes(const bddc_handle* h) { return h ? h->dev_bytes : 0; }

// the persistent solve kernel for a precision, operator form and batch
// (rebalanced over active instances when the batch has several)
const void* solve_kernel_fn(int precision, int formulation, bool bal) {
    if (precision == BDDC_PREC_FP32)
        return bal ? (const void*)bddc_solve_kernel<PrecMixed, true> : (const void*)bddc_solve_kernel<PrecMixed, false>;
    if (formulation == BDDC_FORM_FULL)
        return bal ? (const void*)bddc_solve_kernel<PrecFP64Full, true>
                   : (const void*)bddc_solve_kernel<PrecFP64Full, false>;
    return bal ? (const void*)bddc_solve_kernel<PrecFP64, true> : (const void*)bddc_solve_kernel<PrecFP64, false>;
}

// dense-coarse work units of `rows` rows each: instance, first row, and the
// first unit of every instance (n_inst + 1 entries)
void coarse_units(const Packed& P, int n_inst, int rows, std::vector<int>& cu_inst, std::vector<int>& cu_row0,
                  std::vector<int64_t>& cu0) {
    cu_inst.clear();
    cu_row0.clear();
    cu0.assign(1, 0);
    for (int b = 0; b < n_inst; ++b) {
        for (int64_t r0 = 0; r0 < P.inst_ncn[b]; r0 += rows) {
            cu_inst.push_back(b);
            cu_row0.push_back((int)r0);
        }
        cu0.push_back((int64_t)cu_inst.size());
    }
}

// contiguous subdomain ranges of W warps at equal fractions of the summed
// cost n_Gamma^2 + C: the operators S and F (n_Gamma^2) plus a fixed latency
// cost of a subdomain (gathers, reductions, arrivals); W + 1 entries
std::vector<int64_t> warp_ranges(const Packed& P, int64_t NS, int64_t W, double C) {
    std::vector<double> pre(NS + 1, 0.0);
    for (int64_t s = 0; s < NS; ++s) pre[s + 1] = pre[s] + (double)P.sub_ng[s] * P.sub_ng[s] + C;
    std::vector<int64_t> ws(W + 1);
    int64_t s = 0;
    for (int64_t w = 0; w < W; ++w) {
        const double target = pre[NS] * (double)w / (double)W;
        while (s < NS && pre[s] < target) ++s;
        ws[w] = s;
    }
    ws[W] = NS;
    return ws;
}

// operator-apply units: every subdomain in J = ceil(n_Gamma^2 /
// kDiropPartCost) parts of consecutive outputs (one part in the full-space
// form, whose operator is not a square block); a part's outputs are
// [ob, oe), packed as (ob << 16) | oe
void dirop_units(const Packed& P, int n_inst, bool full, std::vector<int2>& du, std::vector<int64_t>& sub_du0,
                 std::vector<int64_t>& inst_du0) {
    const int64_t NS = (int64_t)P.sub_ng.size();
    du.clear();
    sub_du0.assign(NS + 1, 0);
    for (int64_t s = 0; s < NS; ++s) {
        const int ng = P.sub_ng[s];
        const int64_t cost = (int64_t)ng * ng;
        const int J = full ? 1 : (int)std::max<int64_t>(1, (cost + kDiropPartCost - 1) / kDiropPartCost);
        for (int j = 0; j < J; ++j) {
            const int ob = (int)(((int64_t)ng * j) / J), oe = (int)(((int64_t)ng * (j + 1)) / J);
            du.push_back(make_int2((int)s, (ob << 16) | oe));
        }
        sub_du0[s + 1] = (int64_t)du.size();
    }
    inst_du0.assign(n_inst + 1, 0);
    for (int b = 0; b < n_inst; ++b) inst_du0[b + 1] = sub_du0[P.inst_s1[b]];
}

// contiguous operator-apply unit ranges of W warps at equal fractions of the
// summed cost (outputs x n_Gamma + C); W + 1 entries
std::vector<int64_t> dirop_ranges(const Packed& P, const std::vector<int2>& du, int64_t W, double C) {
    const int64_t NU = (int64_t)du.size();
    std::vector<double> pre(NU + 1, 0.0);
    for (int64_t u = 0; u < NU; ++u) {
        const int ob = du[u].y >> 16, oe = du[u].y & 0xffff;
        pre[u + 1] = pre[u] + (double)(oe - ob) * P.sub_ng[du[u].x] + C;
    }
    std::vector<int64_t> ws(W + 1);
    int64_t u = 0;
    for (int64_t w = 0; w < W; ++w) {
        const double target = pre[NU] * (double)w / (double)W;
        while (u < NU && pre[u] < target) ++u;
        ws[w] = u;
    }
    ws[W] = NU;
    return ws;
}

// launch grid of the persistent kernel: one CTA per subdomain or coarse unit,
// at most the resident CTAs of the device
int solve_grid(int nb, int nsm, int64_t n_sub, int64_t n_cunits) {
    const int64_t want = std::max<int64_t>(n_sub, n_cunits);
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb * nsm, want));
}

constexpr double kBalanceWeight = 4096.0;  // C of the heuristic warp ranges
// tuning probes: launches of kProbeShort and kProbeLong CG iterations give
// the once-per-solve part and the cost per iteration; layouts are compared
// by the predicted time of a kProbeNominal-iteration solve
constexpr int kProbeShort = 2, kProbeLong = 8, kProbeNominal = 30;
constexpr int kProbeRounds = 2;  // rounds over all candidates (minimum per candidate)

// the layouts chosen by earlier tuned setups of this process, by signature
std::mutex g_tune_mu;
std::vector<std::pair<uint64_t, bddc_tuning>> g_tune_cache;

// FNV-1a over what decides the kernel's time per iteration: the launch, the
// subdomains' interface and constraint sizes, the coarse problem
uint64_t tune_signature(const bddc_handle* h, int grid) {
    uint64_t x = 1469598103934665603ULL;
    auto mix = [&](int64_t v) {
        for (int i = 0; i < 8; ++i) {
            x ^= (uint64_t)((v >> (8 * i)) & 0xff);
            x *= 1099511628211ULL;
        }
    };
    const Packed& P = h->P;
    mix(h->precision);
    mix(h->formulation);
    mix(h->n_inst);
    mix(grid);
    mix(P.coarse_sparse ? 1 : 0);
    mix((int64_t)P.sub_ng.size());
    for (size_t s = 0; s < P.sub_ng.size(); ++s) {
        mix(P.sub_ng[s]);
        mix(P.sub_m[s]);
    }
    for (int b = 0; b < h->n_inst; ++b) mix(P.inst_ncn[b]);
    mix((int64_t)P.cn_p.size());
    return x;
}

// device time (ms) of one probe launch of the persistent kernel with the
// layout in p: `iters` CG iterations (tolerance 0) on the handle's constant
// probe data; -1 on a launch error or a barrier timeout
float probe_launch(bddc_handle* h, Params p, int iters) {
    cudaStream_t st = h->stream;
    p.maxit = std::min(iters, p.maxit);  // the CG history's pitch stays within the handle's
    p.tol = 0.0;
    p.f_in = h->d_f;
    p.bc_in = h->d_bc;
    p.flux_out = h->d_flux;
    p.p_out = h->d_p;
    cudaMemsetAsync(p.flux_out, 0, (size_t)h->total_faces * sizeof(double), st);
    cudaMemsetAsync(p.st, 0, sizeof(InstState) * h->n_inst, st);
    cudaMemsetAsync(p.inst_cnt, 0, sizeof(int) * kCounters * (size_t)h->n_inst, st);
    cudaMemsetAsync(p.gsync, 0, sizeof(GridSync), st);
    cudaMemsetAsync(p.tstamp, 0, 2 * sizeof(long long) * (size_t)p.tstamp_cap, st);
    cudaMemcpyAsync(p.n_active, &h->n_inst, sizeof(int), cudaMemcpyHostToDevice, st);
    void* args[] = {&p};
    const void* kfn = solve_kernel_fn(h->precision, h->formulation, p.act_n > 1);
    cudaEventRecord(h->ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel(kfn, dim3(h->grid), dim3(kThreads), args, h->smem, st);
    cudaEventRecord(h->ev1, st);
    if (e != cudaSuccess) return -1.0f;
    cudaMemcpyAsync(h->pin_gs, p.gsync, sizeof(GridSync), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || h->pin_gs->error) return -1.0f;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    return ms;
}

// Autotuning of the work layout (bddc_options.autotune).  Candidates: the
// warp-range weights C and, with the dense coarse solver, the coarse unit
// sizes that leave the launch grid unchanged.  Each candidate is timed by
// probe launches of kProbeShort and kProbeLong iterations, in kProbeRounds
// round-robin rounds after a warm-up (so that a drift of the clocks during
// the tuning favours no candidate), the minimum per candidate and length.
// The predicted time of a kProbeNominal-iteration solve decides; the
// heuristic wins ties within 2 %.  ws_dev is the warp-range buffer
// (grid * kWarps + 1 entries), cu_* the unit buffers, sized for the smallest
// unit.  Returns BDDC_OK or a CUDA error; the handle keeps the heuristic
// layout when a probe fails.
int autotune_layout(bddc_handle* h, int64_t* ws_dev, int* cu_inst_dev, int* cu_row0_dev, int64_t* cu0_dev, int nb,
                    int nsm) {
    const Packed& P = h->P;
    Params& p = h->prm;
    const int64_t NS = P.n_sub, W = (int64_t)h->grid * kWarps;
    const uint64_t sig = tune_signature(h, h->grid);
    bddc_tuning& T = h->tuning;
    std::vector<int> ci, cr;
    std::vector<int64_t> c0;
    auto set_rows = [&](int rows) -> bool {
        coarse_units(P, h->n_inst, rows, ci, cr, c0);
        if (!ci.empty() && (cudaMemcpy(cu_inst_dev, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
                            cudaMemcpy(cu_row0_dev, cr.data(), cr.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
            return false;
        if (cudaMemcpy(cu0_dev, c0.data(), c0.size() * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess) return false;
        p.n_cunits = (int64_t)ci.size();
        p.coarse_rows = rows;
        return true;
    };
    auto set_weight = [&](double C) -> bool {
        const std::vector<int64_t> ws = warp_ranges(P, NS, W, C);
        const std::vector<int64_t> wu = dirop_ranges(P, h->dunit_h, W, C);
        return cudaMemcpy(ws_dev, ws.data(), ws.size() * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(const_cast<int64_t*>(p.warp_du0), wu.data(), wu.size() * sizeof(int64_t),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    };
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& e : g_tune_cache)
            if (e.first == sig) {
                T = e.second;
                T.from_cache = 1;
                break;
            }
    }
    if (T.from_cache) {
        if (!set_weight(T.balance_weight) || !set_rows(T.coarse_rows)) return BDDC_E_CUDA;
        return BDDC_OK;
    }
    // candidates, the heuristic first
    std::vector<std::pair<double, int>> cand;
    const double weights[] = {kBalanceWeight, 0.0, 1024.0, 16384.0, 65536.0};
    std::vector<int> rows_list{kCoarseRows};
    if (!P.coarse_sparse)
        for (int rows : {8, 32}) {
            std::vector<int> a, b;
            std::vector<int64_t> c;
            coarse_units(P, h->n_inst, rows, a, b, c);
            if (solve_grid(nb, nsm, NS, (int64_t)a.size()) == h->grid) rows_list.push_back(rows);
        }
    for (int rows : rows_list)
        for (double C : weights) cand.emplace_back(C, rows);
    cudaMemset(h->d_f, 0x3f, (size_t)h->total_cells * sizeof(double));  // a constant 4.8e-4 in every cell
    cudaMemset(h->d_bc, 0, (size_t)h->total_faces * sizeof(double));
    if (cudaDeviceSynchronize() != cudaSuccess) return BDDC_E_CUDA;
    auto restore = [&]() -> int {
        return set_weight(kBalanceWeight) && set_rows(kCoarseRows) ? BDDC_OK : BDDC_E_CUDA;
    };
    for (int r = 0; r < 3; ++r)  // warm-up
        if (probe_launch(h, p, kProbeLong) < 0.0f) return restore();
    const size_t n = cand.size();
    std::vector<float> t_short(n, 1e30f), t_long(n, 1e30f);
    int cur_rows = kCoarseRows;
    for (int round = 0; round < kProbeRounds; ++round)
        for (size_t k = 0; k < n; ++k) {
            const size_t c = (k + round * (n / 2 + 1)) % n;  // another order each round
            if (!set_weight(cand[c].first)) return BDDC_E_CUDA;
            if (cand[c].second != cur_rows) {
                if (!set_rows(cand[c].second)) return BDDC_E_CUDA;
                cur_rows = cand[c].second;
            }
            const float a = probe_launch(h, p, kProbeShort), b = probe_launch(h, p, kProbeLong);
            if (a < 0.0f || b < 0.0f) return restore();
            t_short[c] = std::min(t_short[c], a);
            t_long[c] = std::min(t_long[c], b);
        }
    auto predict = [&](size_t c) {
        const float per_it = std::max(0.0f, (t_long[c] - t_short[c]) / (float)(kProbeLong - kProbeShort));
        return t_short[c] + (float)(kProbeNominal - kProbeShort) * per_it;
    };
    size_t best = 0;  // the heuristic
    for (size_t c = 1; c < n; ++c)
        if (predict(c) < 0.98f * predict(0) && predict(c) < predict(best)) best = c;
    if (!set_weight(cand[best].first) || !set_rows(cand[best].second)) return BDDC_E_CUDA;
    T.tuned = 1;
    T.balance_weight = cand[best].first;
    T.coarse_rows = cand[best].second;
    T.probe_ms = predict(best);
    T.probe_ms_default = predict(0);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.emplace_back(sig, T);
    return BDDC_OK;
}

// device part of bddc_setup: upload a batch's host setup and size the launch
int setup_from_packed(int n_instances, const bddc_options& opt, void* cuda_stream, Packed&& packed,
                      bddc_handle** out) {
    *out = nullptr;
    bddc_handle* h = new bddc_handle();
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&h->device);
    h->n_inst = n_instances;
    h->maxit = opt.maxit;
    h->precision = opt.precision;
    h->formulation = opt.formulation;
    h->P = std::move(packed);
    Packed& P = h->P;
    for (int b = 0; b < n_instances; ++b) {
        h->total_cells += P.inst_ncells[b];
        h->total_faces += P.inst_nfaces[b];
    }
    // coarse work units (the buffers sized for the smallest unit the tuner tries)
    std::vector<int> cu_inst, cu_row0;
    std::vector<int64_t> cu0;
    coarse_units(P, n_instances, opt.autotune ? 8 : kCoarseRows, cu_inst, cu_row0, cu0);
    // operator-apply units (a part's output range is packed in 16 bits)
    if (P.max_ng > 0xffff) {
        bddc_destroy(h);
        return BDDC_E_INVALID_ARG;
    }
    std::vector<int2> du;
    std::vector<int64_t> sub_du0, inst_du0;
    dirop_units(P, n_instances, opt.formulation == BDDC_FORM_FULL, du, sub_du0, inst_du0);
    h->dunit_h = du;
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
    UP(cunit_inst, cu_inst); UP(cunit_row0, cu_row0); UP(inst_cu0, cu0);
    UP(dunit, du); UP(sub_du0, sub_du0); UP(inst_du0, inst_du0);
    if (opt.formulation == BDDC_FORM_FULL) {
        UP(slot_fk, P.slot_fk); UP(slot_fopp, P.slot_fopp); UP(slot_fcell, P.slot_fcell);
    }
    UP(Gpre, P.Gpre); UP(P64, P.P64);
    if (P.dev_Gpost) {  // computed on the device by the setup: adopted, freed with the handle's Packed
        p.Gpost = P.dev_Gpost.get();
        h->dev_bytes += sizeof(double) * (size_t)P.dev_Gpost_count;
    } else {
        UP(Gpost, P.Gpost);
    }
    UP(slot_fcs, P.slot_fcs); UP(cslot_n, P.cslot_n); UP(slot_coef, P.slot_coef);
    UP(slot_fperm, P.slot_fperm); UP(cslot_fstart, P.cslot_fstart); UP(slot_fcoefp, P.slot_fcoefp);
    {
        auto pairs2 = [](const std::vector<double>& v) {
            std::vector<float2> o(v.size());
            for (size_t q = 0; q < v.size(); ++q) {
                const float hi = (float)v[q];
                o[q] = make_float2(hi, (float)(v[q] - (double)hi));
            }
            return o;
        };
        std::vector<double> invn(P.cslot_n.size(), 0.0);
        for (size_t q = 0; q < invn.size(); ++q) invn[q] = P.cslot_n[q] > 0 ? 1.0 / P.cslot_n[q] : 0.0;
        std::vector<float> cf(P.slot_coef.begin(), P.slot_coef.end()), cfp(P.slot_fcoefp.begin(), P.slot_fcoefp.end());
        if (!rc) rc = upload(h, pairs2(P.slot_w), &p.slot_w2);
        if (!rc) rc = upload(h, pairs2(P.slot_dsig), &p.slot_dsig2);
        if (!rc) rc = upload(h, pairs2(invn), &p.cslot_inv2);
        if (!rc) rc = upload(h, cf, &p.slot_coef_f);
        if (!rc) rc = upload(h, cfp, &p.slot_fcoefp_f);
    }
    UP(inst_cfoff, h->inst_cfoff);
    UP(inst_grid, P.inst_grid); UP(inst_h, P.inst_h); UP(cell_kinv, P.cell_kinv); UP(face_bct, P.face_bct);
    UP(inst_face_off, P.inst_face_off); UP(inst_cell_off, P.inst_cell_off);
    if (!rc && P.coarse_sparse) {
        // multifrontal coarse factor and its work units per tree depth
        p.coarse_sparse = 1;
        UP(inst_csoff, P.inst_csoff);
        UP(cn_X, P.cn_X); UP(cn_H, P.cn_H); UP(cn_HT, P.cn_HT);
        const int L = P.cn_max_depth + 1;
        const size_t nn = P.cn_p.size();
        // the sweep units hold 32-bit offsets
        const int64_t kLim = (int64_t)1 << 31;
        if ((int64_t)P.cn_X.size() >= kLim || (int64_t)P.cn_H.size() >= kLim || (int64_t)P.cn_dof.size() >= kLim ||
            P.n_csys >= kLim || P.n_cu >= kLim) {
            bddc_destroy(h);
            return BDDC_E_INVALID_ARG;  // coarse factor too large for one handle
        }
        // per front position: (dof, c0, c1, -)
        {
            std::vector<int4> idx(P.cn_dof.size());
            for (size_t q = 0; q < idx.size(); ++q) idx[q] = make_int4(P.cn_dof[q], P.cn_c0[q], P.cn_c1[q], 0);
            UP(cn_idx, idx);
        }
        std::vector<std::vector<CsUnit>> fw(L), bw(L);
        std::vector<int64_t> fwc(nn), fwp(nn), bwc(nn), bwp(nn);
        int64_t nfc = 0, nfp = 0, nbc = 0, nbp = 0;
        for (size_t v = 0; v < nn; ++v) {
            const int d = P.cn_depth[v], pp = P.cn_p[v], q = P.cn_q[v], b = P.cn_inst[v];
            const int ncb = std::max(1, (q + 31) / 32), nic = pp > 0 ? (pp + kCsChunk - 1) / kCsChunk : 1;
            const int nrb = (pp + 31) / 32, nkc = (pp + q + kCsChunk - 1) / kCsChunk;
            fwc[v] = nfc; nfc += ncb;
            fwp[v] = nfp; nfp += (int64_t)ncb * nic * 32;
            bwc[v] = nbc; nbc += nrb;
            bwp[v] = nbp; nbp += (int64_t)nrb * nkc * 32;
            CsUnit U{};
            U.pp = pp; U.q = q; U.b = b;
            U.od = (int)P.cn_off_dof[v];
            U.cs = (int)P.inst_csoff[b];
            for (int cb = 0; cb < ncb; ++cb)
                for (int ic = 0; ic < nic; ++ic) {
                    U.blk = cb; U.ich = ic; U.nch = nic;
                    U.k0 = std::min(pp, ic * kCsChunk);
                    U.k1 = std::min(pp, U.k0 + kCsChunk);
                    U.om = (int)P.cn_off_H[v];
                    U.ou = (int)P.cn_off_u[v];
                    U.pof = (int)(fwp[v] + (int64_t)cb * nic * 32);
                    U.cof = (int)(fwc[v] + cb);
                    fw[d].push_back(U);
                }
            for (int rb = 0; rb < nrb; ++rb)
                for (int kc = 0; kc < nkc; ++kc) {
                    U.blk = rb; U.ich = kc; U.nch = nkc;
                    U.k0 = kc * kCsChunk;
                    U.k1 = std::min(pp + q, U.k0 + kCsChunk);
                    U.om = (int)P.cn_off_X[v];
                    U.ou = (int)P.cn_off_H[v];
                    U.pof = (int)(bwp[v] + (int64_t)rb * nkc * 32);
                    U.cof = (int)(bwc[v] + rb);
                    bw[d].push_back(U);
                }
        }
        if (!rc) rc = dalloc(h, (size_t)std::max<int64_t>(nfc, 1), &p.cs_fcnt);
        if (!rc) rc = dalloc(h, (size_t)std::max<int64_t>(nbc, 1), &p.cs_bcnt);
        if (!rc) rc = dalloc(h, (size_t)std::max<int64_t>(nfp, 1), &p.cs_fpart);
        if (!rc) rc = dalloc(h, (size_t)std::max<int64_t>(nbp, 1), &p.cs_bpart);
        std::vector<CsUnit> fu, bu;
        std::vector<int64_t> fo(1, 0), bo(1, 0);
        for (int d = 0; d < L; ++d) {
            fu.insert(fu.end(), fw[d].begin(), fw[d].end());
            bu.insert(bu.end(), bw[d].begin(), bw[d].end());
            fo.push_back((int64_t)fu.size());
            bo.push_back((int64_t)bu.size());
        }
        UP(fw_unit, fu); UP(bw_unit, bu); UP(fw_off, fo); UP(bw_off, bo);
        h->fw_off_h = fo;
        h->bw_off_h = bo;
        p.cn_levels = L;
    }
#undef UP
    if (!rc) {
        if (opt.precision == BDDC_PREC_FP32) {
            // S and the coarse inverse as FP32 pairs (hi, lo); F and Psi FP32.
            // The conversion runs on the setup's host threads (GBs for large
            // batches).
            const int nth = opt.n_threads > 0 ? opt.n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
            auto pairs = [nth](const std::vector<double>& v) {
                std::vector<float2> o(v.size());
                const size_t n = v.size();
                const size_t T = (size_t)std::max<int64_t>(1, std::min<int64_t>(nth, (int64_t)(n >> 16) + 1));
                std::vector<std::thread> th;
                for (size_t t = 0; t < T; ++t)
                    th.emplace_back([&v, &o, n, T, t] {
                        for (size_t q = n * t / T; q < n * (t + 1) / T; ++q) {
                            const float hi = (float)v[q];
                            o[q] = make_float2(hi, (float)(v[q] - (double)hi));
                        }
                    });
                for (std::thread& x : th) x.join();
                return o;
            };
            const float *f = nullptr, *pp = nullptr;
            const float2 *k2 = nullptr, *s2 = nullptr;
            rc = upload(h, P.F32, &f);
            if (!rc) rc = upload(h, P.P32, &pp);
            if (!rc) rc = upload(h, pairs(P.S), &s2);
            if (!rc) rc = upload(h, pairs(P.Kinv), &k2);
            if (!rc) {
                if (P.dev_Gpost) {
                    // written in full by k_pairs on the handle's stream: no zeroing
                    float2* g2 = nullptr;
                    if (cudaMalloc((void**)&g2, std::max<int64_t>(P.dev_Gpost_count, 1) * sizeof(float2)) != cudaSuccess) {
                        cudaGetLastError();
                        rc = BDDC_E_OOM;
                    } else {
                        h->allocs.push_back(g2);
                        h->dev_bytes += sizeof(float2) * (size_t)P.dev_Gpost_count;
                    }
                    if (!rc) {
                        const int64_t cnt = P.dev_Gpost_count;
                        k_pairs<<<(int)std::min<int64_t>((cnt + 255) / 256, 65536), 256, 0, h->stream>>>(cnt, p.Gpost, g2);
                        if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = BDDC_E_CUDA;
                    }
                    p.Gpost2 = g2;
                } else {
                    rc = upload(h, pairs(P.Gpost), &p.Gpost2);
                }
            }
            p.F = f;
            p.P = pp;
            p.S = s2;
            p.Kinv = k2;
        } else {
            const double *f = nullptr, *s64 = nullptr, *k64 = nullptr;
            rc = upload(h, P.F64, &f);
            if (!rc) rc = upload(h, P.S, &s64);
            if (!rc) rc = upload(h, P.Kinv, &k64);
            p.F = f;
            p.P = p.P64;
            p.S = s64;
            p.Kinv = k64;
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
    AL(part_dq, (int64_t)du.size()); AL(part_rr, NS); AL(part_rz, NS); AL(part_a1, NS); AL(part_a2, NS);
    AL(inst_cnt, (size_t)n_instances * kCounters); AL(inst_tot, (size_t)n_instances * kTotals);
    AL(st, n_instances); AL(alpha_hist, H); AL(beta_hist, H); AL(rho_hist, H);
    AL(n_active, 1); AL(gsync, 1);
    AL(tr_part, (size_t)n_instances * kTrChunks * 4); AL(tr_out, n_instances);
    if (P.coarse_sparse) {
        AL(cs_b, P.n_csys); AL(cs_t, P.n_csys); AL(cs_x, P.n_csys); AL(cs_u, std::max<int64_t>(P.n_cu, 1));
    }
    p.tstamp_cap = 16 + 4 * (opt.maxit + 2);
    AL(tstamp, 2 * (size_t)p.tstamp_cap);
#undef AL
    if (rc) {
        bddc_destroy(h);
        return rc;
    }
    p.n_inst = n_instances;
    p.n_sub = NS;
    p.n_du = (int64_t)du.size();
    if (opt.autotune) coarse_units(P, n_instances, kCoarseRows, cu_inst, cu_row0, cu0);
    if (!cu_inst.empty() && opt.autotune) {  // the default units into the larger buffers
        cudaMemcpy(const_cast<int*>(p.cunit_inst), cu_inst.data(), cu_inst.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(const_cast<int*>(p.cunit_row0), cu_row0.data(), cu_row0.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(const_cast<int64_t*>(p.inst_cu0), cu0.data(), cu0.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    }
    p.n_cunits = (int64_t)cu_inst.size();
    p.coarse_rows = kCoarseRows;
    p.maxit = opt.maxit;
    p.max_ng = std::max(P.max_ng, 1);
    p.max_in_post = std::max(P.max_in_post, 1);
    p.max_ncn = P.coarse_sparse ? 2 : std::max(P.max_ncn, 1);  // the CTA rhs area of the dense coarse solve
    p.max_m = std::max(P.max_m, 1);
    p.max_ext = opt.formulation == BDDC_FORM_FULL ? std::max(P.max_out_post, 1) : 0;
    p.act_n = n_instances <= kActMaxInst ? n_instances : 0;
    h->smem = sizeof(double) * ((size_t)p.max_ncn + (size_t)kWarps * (2 * (size_t)p.max_ng + p.max_in_post +
                                                                       2 * ((size_t)p.max_m + 1) + p.max_ext)) +
              sizeof(int) * 2 * ((size_t)p.act_n + 1);
    if (h->smem > 200 * 1024) {
        // the CTA's dense coarse right-hand side plus 8 warp areas (each with
        // the largest subdomain's interior fluxes and cells for the
        // post-correction) must fit one CTA's shared memory
        g_setup_err = "shared memory per CTA (" + std::to_string(h->smem / 1024) +
                      " KB) above 200 KB: the dense coarse problem or a subdomain's interior is too large";
        bddc_destroy(h);
        return BDDC_E_INVALID_ARG;
    }
    const void* kfn = solve_kernel_fn(opt.precision, opt.formulation, p.act_n > 1);
    // the stand-alone operator / preconditioner kernels use the same carve
    const void* aux[] = {(const void*)k_operator_local<PrecFP64>, (const void*)k_operator_local<PrecMixed>,
                         (const void*)k_precond_restrict<PrecFP64>, (const void*)k_precond_restrict<PrecMixed>,
                         (const void*)k_precond_coarse<PrecFP64>, (const void*)k_precond_coarse<PrecMixed>,
                         (const void*)k_precond_prolong<PrecFP64>, (const void*)k_precond_prolong<PrecMixed>};
    bool attr_ok = ensure_smem(kfn, h->smem);
    for (const void* f : aux) attr_ok = attr_ok && ensure_smem(f, h->smem);
    if (!attr_ok) {
        cudaGetLastError();
        bddc_destroy(h);
        return BDDC_E_CUDA;
    }
    int nb = 0, nsm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, kThreads, h->smem);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
    h->grid = solve_grid(nb, nsm, NS, p.n_cunits);
    if (nb <= 0) {
        bddc_destroy(h);
        return BDDC_E_CUDA;
    }
    {
        // warp ranges at the heuristic weight C = 4096, a fixed cost worth a
        // 64-dof interface.  Measured on GB300: the irregular 3-8-cell boxes
        // of the 60x220x85 grid 153 -> 109 ms per solve against equal
        // subdomain counts; pure n_Gamma^2 made the regular partitions
        // 3-13 % slower, this weight within 1 %.
        const int64_t* d = nullptr;
        const int64_t* dd = nullptr;
        if (upload(h, warp_ranges(P, NS, (int64_t)h->grid * kWarps, kBalanceWeight), &d) != BDDC_OK ||
            upload(h, dirop_ranges(P, h->dunit_h, (int64_t)h->grid * kWarps, kBalanceWeight), &dd) != BDDC_OK) {
            bddc_destroy(h);
            return BDDC_E_OOM;
        }
        p.warp_sub0 = d;
        p.warp_du0 = dd;
    }
    h->tuning.balance_weight = kBalanceWeight;
    h->tuning.coarse_rows = kCoarseRows;
    cudaEventCreate(&h->ev0);
    cudaEventCreate(&h->ev1);
    if (cudaMallocHost((void**)&h->pin_st, sizeof(InstState) * n_instances) != cudaSuccess ||
        cudaMallocHost((void**)&h->pin_tr, sizeof(double) * n_instances) != cudaSuccess ||
        cudaMallocHost((void**)&h->pin_gs, sizeof(GridSync)) != cudaSuccess) {
        bddc_destroy(h);
        return BDDC_E_OOM;
    }
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
    // (the mixed path stores S and the coarse inverse as FP32 pairs: 8 bytes)
    const double fb = opt.precision == BDDC_PREC_FP32 ? 4.0 : 8.0;
    double it_b = 0.0, pre_b = 0.0, post_b = 0.0;
    for (int64_t s = 0; s < NS; ++s) {
        const double ng = P.sub_ng[s], m = P.sub_m[s], nc = P.sub_nc[s], ni = P.sub_ni[s];
        // the operator: S^i, or in the full form the extension's n_Gamma
        // columns of G_post and the per-slot face data (16 bytes)
        const double op_b = opt.formulation == BDDC_FORM_FULL ? 8.0 * ng * (ni + nc) + 16.0 * ng : 8.0 * ng * ng;
        it_b += op_b + fb * ng * ng + 2.0 * fb * m * ng + 8.0 * 18.0 * ng;
        // the source columns of G_pre and G_post are not counted: they are
        // skipped for source-free subdomains
        pre_b += 3.0 * fb * m * ng + 8.0 * ng * ng + fb * ng * ng + 8.0 * 20.0 * ng;
        post_b += 8.0 * ng * (ni + nc) + 8.0 * (ni + 2.0 * nc + 2.0 * ng);
    }
    if (P.coarse_sparse) {
        // a sparse coarse solve reads X, H (forward) and H^T (backward) once
        double cb = 0.0;
        for (size_t v = 0; v < P.cn_p.size(); ++v)
            cb += 8.0 * ((double)P.cn_p[v] * P.cn_p[v] + 2.0 * P.cn_p[v] * P.cn_q[v]);
        it_b += cb;
        pre_b += 2.0 * cb;
    } else {
        for (int b = 0; b < n_instances; ++b) {
            const double ncn = P.inst_ncn[b], ncf = P.inst_ncf[b];
            it_b += 8.0 * ncn * ncf;
            pre_b += 8.0 * ncn * ncn + 8.0 * ncn * ncf;
        }
    }
    h->bytes_iter = it_b;
    h->bytes_pre = pre_b;
    h->bytes_post = post_b;
    // the uploads and the zeroing of the work vectors ran on the legacy
    // default stream; a non-blocking solve stream does not wait for it
    if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        bddc_destroy(h);
        return BDDC_E_CUDA;
    }
    if (opt.autotune) {
        // the probes' constant data live in the staging buffers of bddc_solve
        if (dalloc(h, (size_t)h->total_cells, &h->d_f) || dalloc(h, (size_t)h->total_faces, &h->d_bc) ||
            dalloc(h, (size_t)h->total_faces, &h->d_flux) || dalloc(h, (size_t)h->total_cells, &h->d_p)) {
            bddc_destroy(h);
            return BDDC_E_OOM;
        }
        if (autotune_layout(h, const_cast<int64_t*>(p.warp_sub0), const_cast<int*>(p.cunit_inst),
                            const_cast<int*>(p.cunit_row0), const_cast<int64_t*>(p.inst_cu0), nb, nsm) != BDDC_OK ||
            cudaGetLastError() != cudaSuccess) {
            bddc_destroy(h);
            return BDDC_E_CUDA;
        }
    }
    *out = h;
    return BDDC_OK;
}

}  // namespace bddc

extern "C" {

int bddc_sizes(const bddc_handle* h, int* n_instances, int64_t* n_interface, int64_t* n_subdomains) {
    if (!h) return BDDC_E_INVALID_ARG;
    if (n_instances) *n_instances = h->n_inst;
    if (n_interface) *n_interface = h->P.n_gamma;
    if (n_subdomains) *n_subdomains = h->P.n_sub;
    return BDDC_OK;
}

int bddc_get_tuning(const bddc_handle* h, bddc_tuning* out) {
    if (!h || !out) return BDDC_E_INVALID_ARG;
    *out = h->tuning;
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
        if (std::find(h->allocs.begin(), h->allocs.end(), (void*)*buf) == h->allocs.end()) {
            h->allocs.push_back(*buf);
            h->dev_bytes += n * sizeof(double);
        }
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
    cudaMemsetAsync(p.inst_cnt, 0, sizeof(int) * kCounters * (size_t)h->n_inst, st);
    cudaMemsetAsync(p.gsync, 0, sizeof(GridSync), st);
    cudaMemsetAsync(p.tstamp, 0, 2 * sizeof(long long) * (size_t)p.tstamp_cap, st);
    cudaMemcpyAsync(p.n_active, &h->n_inst, sizeof(int), cudaMemcpyHostToDevice, st);
    void* args[] = {&p};
    const void* kfn = solve_kernel_fn(h->precision, h->formulation, p.act_n > 1);
    cudaEventRecord(h->ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel(kfn, dim3(h->grid), dim3(kThreads), args, h->smem, st);
    cudaEventRecord(h->ev1, st);
    if (e != cudaSuccess) return set_err(h, BDDC_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    // the true residual of the full system at the solution
    k_true_residual<<<h->n_inst * kTrChunks, kThreads, 0, st>>>(p);
    k_true_residual_sum<<<(h->n_inst + 127) / 128, 128, 0, st>>>(p);
    cudaMemcpyAsync(h->pin_tr, p.tr_out, sizeof(double) * h->n_inst, cudaMemcpyDeviceToHost, st);
    if (!flux_dev) cudaMemcpyAsync(flux, p.flux_out, nface * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!p_dev) cudaMemcpyAsync(pressure, p.p_out, ncell * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h->pin_st, p.st, sizeof(InstState) * h->n_inst, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h->pin_gs, p.gsync, sizeof(GridSync), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(h, BDDC_E_CUDA, std::string("solve: ") + cudaGetErrorString(e));
    const InstState* hs = h->pin_st;
    const GridSync& gs = *h->pin_gs;
    cudaEventElapsedTime(&h->last_ms, h->ev0, h->ev1);
    if (gs.error) return set_err(h, BDDC_E_TIMEOUT, "grid barrier wait exceeded its limit");
    int ret = BDDC_OK;
    double total_it = 0.0;
    int max_it = 0;
    std::vector<int> its_h(h->n_inst);
    for (int b = 0; b < h->n_inst; ++b) {
        bddc_stats& S = h->stats[b];
        S.iterations = hs[b].iterations;
        S.status = hs[b].done ? hs[b].status : BDDC_E_TIMEOUT;
        S.relres = hs[b].relres;
        S.true_relres = h->pin_tr[b];
        const int m = S.iterations;
        S.kappa = 0.0;  // computed on demand from the CG coefficients
        its_h[b] = S.iterations;
        if (S.status != BDDC_OK && ret == BDDC_OK) ret = S.status;
        total_it += m;
        max_it = std::max(max_it, m);
    }
    if (iterations) {  // one copy for the whole batch
        if (is_device_ptr(iterations)) {
            cudaMemcpyAsync(iterations, its_h.data(), sizeof(int) * its_h.size(), cudaMemcpyHostToDevice, st);
            cudaStreamSynchronize(st);
        } else {
            std::copy(its_h.begin(), its_h.end(), iterations);
        }
    }
    // work of the kernel: every instance runs its own iterations; the
    // persistent loop streams only active instances' operators
    h->last_bytes = h->bytes_pre + h->bytes_post + h->bytes_iter * (total_it / std::max(1, h->n_inst));
    h->kappa_stale = true;
    if (ret != BDDC_OK) set_err(h, ret, "one or more instances did not converge");
    return ret;
}

namespace {
// Lanczos estimate of the condition number from the CG coefficients of the
// last solve (Sec. 5): extreme eigenvalues of the tridiagonal matrix built
// from alpha and beta.  Fetches the used columns of the coefficient history.
void compute_kappa(const bddc_handle* h) {
    int hist_cols = 1;
    for (int b = 0; b < h->n_inst; ++b) hist_cols = std::max(hist_cols, std::min(h->stats[b].iterations, h->maxit) + 1);
    const size_t pitch = sizeof(double) * (size_t)(h->maxit + 1);
    std::vector<double>& ha = h->hist_a;
    std::vector<double>& hb = h->hist_b;
    if (ha.size() != (size_t)h->n_inst * (h->maxit + 1)) {
        ha.assign((size_t)h->n_inst * (h->maxit + 1), 0.0);
        hb.assign((size_t)h->n_inst * (h->maxit + 1), 0.0);
    }
    cudaMemcpy2D(ha.data(), pitch, h->prm.alpha_hist, pitch, sizeof(double) * hist_cols, h->n_inst,
                 cudaMemcpyDeviceToHost);
    cudaMemcpy2D(hb.data(), pitch, h->prm.beta_hist, pitch, sizeof(double) * hist_cols, h->n_inst,
                 cudaMemcpyDeviceToHost);
    for (int b = 0; b < h->n_inst; ++b) {
        bddc_stats& S = h->stats[b];
        const int m = S.iterations;
        S.kappa = 1.0;
        if (m <= 0) continue;
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
    h->kappa_stale = false;
}
}  // namespace

int bddc_debug_vector(const bddc_handle* h, const char* name, double* dst, int64_t* count) {
    if (!h || !name) return BDDC_E_INVALID_ARG;
    const Params& p = h->prm;
    const std::string n(name);
    const int64_t G = h->P.n_gamma, L = h->P.off_slot.back(), CL = h->P.off_cslot.back(), NS = h->P.n_sub;
    const double* src = nullptr;
    int64_t len = 0;
    if (n == "x") { src = p.x; len = G; }
    else if (n == "r0") { src = p.rbuf0; len = G; }
    else if (n == "r1") { src = p.rbuf1; len = G; }
    else if (n == "d0") { src = p.dbuf0; len = G; }
    else if (n == "d1") { src = p.dbuf1; len = G; }
    else if (n == "g") { src = p.g; len = G; }
    else if (n == "u0") { src = p.u0; len = G; }
    else if (n == "ql") { src = p.ql; len = L; }
    else if (n == "zl") { src = p.zl; len = L; }
    else if (n == "yl") { src = p.yl; len = L; }
    else if (n == "rl") { src = p.rl; len = L; }
    else if (n == "tl") { src = p.tl; len = L; }
    else if (n == "rcl") { src = p.rcl; len = CL; }
    else if (n == "wc") { src = p.wc; len = h->P.n_coarse_vec; }
    else if (n == "xp") { src = p.xp; len = NS; }
    else if (n == "zp") { src = p.zp; len = NS; }
    else if (n == "prhs") { src = p.prhs; len = NS; }
    else if (n == "part_rr") { src = p.part_rr; len = NS; }
    else if (n == "part_rz") { src = p.part_rz; len = NS; }
    else if (n == "part_dq") { src = p.part_dq; len = p.n_du; }
    else if (n == "alpha") { src = p.alpha_hist; len = (int64_t)h->n_inst * (p.maxit + 1); }
    else if (n == "beta") { src = p.beta_hist; len = (int64_t)h->n_inst * (p.maxit + 1); }
    else return BDDC_E_INVALID_ARG;
    if (count) *count = len;
    if (dst && len) {
        if (cudaMemcpy(dst, src, len * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return BDDC_E_CUDA;
    }
    return BDDC_OK;
}

int bddc_debug_phase_times(const bddc_handle* h, int64_t* pairs, int64_t* count) {
    if (!h) return BDDC_E_INVALID_ARG;
    const int64_t n = 2 * (int64_t)h->prm.tstamp_cap;
    if (count) *count = n;
    if (pairs && cudaMemcpy(pairs, h->prm.tstamp, n * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return BDDC_E_CUDA;
    return BDDC_OK;
}

int bddc_debug_barrier_timeout(long long limit_ns, int n_ctas) {
    if (limit_ns <= 0 || limit_ns > 60000000000LL || n_ctas < 2 || n_ctas > 1024) return BDDC_E_INVALID_ARG;
    GridSync* gs = nullptr;
    if (cudaMalloc((void**)&gs, sizeof(GridSync)) != cudaSuccess) {
        cudaGetLastError();
        return BDDC_E_CUDA;
    }
    cudaMemset(gs, 0, sizeof(GridSync));
    k_barrier_probe<<<n_ctas, 32>>>(gs, limit_ns);
    GridSync hgs{};
    const cudaError_t e = cudaMemcpy(&hgs, gs, sizeof(GridSync), cudaMemcpyDeviceToHost);
    cudaFree(gs);
    if (e != cudaSuccess) return BDDC_E_CUDA;
    return hgs.error ? BDDC_E_TIMEOUT : BDDC_OK;
}

int bddc_get_stats(const bddc_handle* h, int instance, bddc_stats* out) {
    if (!h || !out || instance < 0 || instance >= h->n_inst) return BDDC_E_INVALID_ARG;
    if (h->kappa_stale) compute_kappa(h);
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
    const int grid = (int)std::min<int64_t>((p.n_sub + kWarps - 1) / kWarps, 4096);
    if (h->precision == BDDC_PREC_FP32) k_operator_local<PrecMixed><<<grid, kThreads, h->smem, h->stream>>>(p, u, p0);
    else k_operator_local<PrecFP64><<<grid, kThreads, h->smem, h->stream>>>(p, u, p0);
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
    const int grid = (int)std::min<int64_t>((p.n_sub + kWarps - 1) / kWarps, 4096);
    const int cgrid = (int)std::min<int64_t>(p.n_cunits, 4096);
    // the stand-alone kernels keep the coarse vectors in FP64 on both paths,
    // so the sparse sweeps run in their FP64 instantiation
    auto coarse = [&](bool mixed) {
        if (p.coarse_sparse) {
            const int igrid = (int)std::min<int64_t>((h->P.n_csys + kThreads - 1) / kThreads, 4096);
            k_cs_rhs<PrecFP64><<<igrid, kThreads, 0, h->stream>>>(p);
            for (int d = p.cn_levels - 1; d >= 0; --d) {
                const int64_t nu = h->fw_off_h[d + 1] - h->fw_off_h[d];
                if (nu > 0) k_cs_forward<<<(int)std::min<int64_t>((nu + kWarps - 1) / kWarps, 4096), kThreads, 0, h->stream>>>(p, d);
            }
            for (int d = 0; d < p.cn_levels; ++d) {
                const int64_t nu = h->bw_off_h[d + 1] - h->bw_off_h[d];
                if (nu > 0)
                    k_cs_backward<PrecFP64><<<(int)std::min<int64_t>((nu + kWarps - 1) / kWarps, 4096), kThreads, 0, h->stream>>>(p, d);
            }
        } else if (mixed) {
            k_precond_coarse<PrecMixed><<<cgrid, kThreads, h->smem, h->stream>>>(p);
        } else {
            k_precond_coarse<PrecFP64><<<cgrid, kThreads, h->smem, h->stream>>>(p);
        }
    };
    if (h->precision == BDDC_PREC_FP32) {
        k_precond_restrict<PrecMixed><<<grid, kThreads, h->smem, h->stream>>>(p, r);
        coarse(true);
        k_precond_prolong<PrecMixed><<<grid, kThreads, h->smem, h->stream>>>(p, z0);
    } else {
        k_precond_restrict<PrecFP64><<<grid, kThreads, h->smem, h->stream>>>(p, r);
        coarse(false);
        k_precond_prolong<PrecFP64><<<grid, kThreads, h->smem, h->stream>>>(p, z0);
    }
    const int64_t L = h->P.off_slot.back();
    k_assemble<<<(int)std::min<int64_t>((L + 255) / 256, 4096), 256, 0, h->stream>>>(L, p.zl, p.slot_g, p.slot_partner, z);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? BDDC_OK : set_err(h, BDDC_E_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

namespace {
// Sizes of a raw subassembled apply, read on the caller's stream (so that
// work queued there before the call, which may write the tables, is
// finished) and validated: every local size 0..1024, slot_offset[0] = 0 and
// slot_offset[s + 1] - slot_offset[s] = ng[s] (consecutive, non-overlapping
// slot ranges), the total at most max_slots.  Returns BDDC_OK with the
// total in *n_slots, or an error code with the message in *msg.
int raw_apply_sizes(int n_sub, const int* ng, const int64_t* slot_offset, cudaStream_t st, int64_t max_slots,
                    int64_t* n_slots, std::string* msg) {
    std::vector<int> hng((size_t)n_sub);
    std::vector<int64_t> hoff((size_t)n_sub + 1);
    cudaError_t e = cudaMemcpyAsync(hng.data(), ng, sizeof(int) * (size_t)n_sub, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hoff.data(), slot_offset, sizeof(int64_t) * ((size_t)n_sub + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *msg = std::string("reading the sizes: ") + cudaGetErrorString(e);
        return BDDC_E_CUDA;
    }
    if (hoff[0] != 0) {
        *msg = "slot_offset[0] must be 0";
        return BDDC_E_INVALID_ARG;
    }
    for (int s = 0; s < n_sub; ++s) {
        if (hng[s] < 0 || hng[s] > 1024) {
            *msg = "local interface size " + std::to_string(hng[s]) + " of subdomain " + std::to_string(s) +
                   " is outside 0..1024";
            return BDDC_E_INVALID_ARG;
        }
        if (hoff[s + 1] - hoff[s] != hng[s]) {
            *msg = "slot_offset is not the prefix sum of ng at subdomain " + std::to_string(s);
            return BDDC_E_INVALID_ARG;
        }
    }
    *n_slots = hoff[n_sub];
    if (*n_slots > max_slots) {
        *msg = std::to_string(*n_slots) + " local slots exceed the fixed scratch of " + std::to_string(max_slots) +
               " doubles; use bddc_subassembled_apply with caller scratch";
        return BDDC_E_INVALID_ARG;
    }
    return BDDC_OK;
}
}  // namespace

extern "C" {

int bddc_subassembled_apply(int n_sub, const int* ng, const int64_t* slot_offset, const int64_t* S_offset,
                            const double* S, const int* gidx, const int* partner, int64_t n_interface,
                            const double* u, double* q, double* slot_scratch, void* stream) {
    g_setup_err.clear();
    if (n_sub <= 0 || !ng || !slot_offset || !S_offset || !S || !gidx || !partner || !u || !q || !slot_scratch ||
        n_interface <= 0) {
        g_setup_err = "bddc_subassembled_apply: null pointer or non-positive size";
        return BDDC_E_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t n_slots = 0;
    std::string msg;
    const int rc = raw_apply_sizes(n_sub, ng, slot_offset, st, INT32_MAX, &n_slots, &msg);
    if (rc) {
        g_setup_err = "bddc_subassembled_apply: " + msg;
        return rc;
    }
    cudaGetLastError();  // an earlier, unrelated launch error is not this call's
    k_subassembled_local<<<std::min(n_sub, 4096), 128, 0, st>>>(n_sub, ng, slot_offset, S_offset, S, gidx, u,
                                                                slot_scratch, n_slots, n_interface);
    k_assemble_checked<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_slots + 255) / 256, 4096)), 256, 0, st>>>(
        n_slots, slot_scratch, gidx, partner, n_interface, q);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_setup_err = std::string("bddc_subassembled_apply: launch: ") + cudaGetErrorString(e);
        return BDDC_E_CUDA;
    }
    return BDDC_OK;
}

}  // extern "C"

// ---- allocation-free subassembled apply -------------------------------------------
// The scratch of bddc_subassembled_apply_noalloc: one fixed array of the
// library's device memory.  Host code never dereferences this name (on the
// host it is only a stand-in for the symbol); its device address is looked
// up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[BDDC_NOALLOC_MAX_SLOTS];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (looked up on
// the first call per device)
int noalloc_scratch(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return BDDC_E_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return BDDC_E_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(ptr);
    }
    *out = g_noalloc_ptr[dev];
    return BDDC_OK;
}
}  // namespace

extern "C" int bddc_subassembled_apply_noalloc(int n_sub, const int* ng, const int64_t* slot_offset,
                                               const int64_t* S_offset, const double* S, const int* gidx,
                                               const int* partner, int64_t n_interface, const double* u,
                                               double* q, void* stream) {
    g_setup_err.clear();
    if (n_sub <= 0 || !ng || !slot_offset || !S_offset || !S || !gidx || !partner || !u || !q || n_interface <= 0) {
        g_setup_err = "bddc_subassembled_apply_noalloc: null pointer or non-positive size";
        return BDDC_E_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t n_slots = 0;
    std::string msg;
    int rc = raw_apply_sizes(n_sub, ng, slot_offset, st, (int64_t)BDDC_NOALLOC_MAX_SLOTS, &n_slots, &msg);
    if (rc) {
        g_setup_err = "bddc_subassembled_apply_noalloc: " + msg;
        return rc;
    }
    double* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) {
        g_setup_err = "bddc_subassembled_apply_noalloc: cudaGetSymbolAddress failed";
        return rc;
    }
    cudaGetLastError();  // an earlier, unrelated launch error is not this call's
    // the kernels' index checks use n_slots (at most the array's size), so
    // no access leaves the fixed array, whatever the caller's tables hold
    k_subassembled_local<<<std::min(n_sub, 4096), 128, 0, st>>>(n_sub, ng, slot_offset, S_offset, S, gidx, u, scratch,
                                                                n_slots, n_interface);
    k_assemble_checked<<<(int)std::max<int64_t>(1, std::min<int64_t>((n_slots + 255) / 256, 4096)), 256, 0, st>>>(
        n_slots, scratch, gidx, partner, n_interface, q);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_setup_err = std::string("bddc_subassembled_apply_noalloc: launch: ") + cudaGetErrorString(e);
        return BDDC_E_CUDA;
    }
    return BDDC_OK;
}

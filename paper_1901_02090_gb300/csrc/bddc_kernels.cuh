// Device-side data layout of the BDDC solve.
//
// One persistent cooperative kernel runs Algorithm 1 of the paper for every
// instance of a batch: Step 1 (coarse solve), Step 2 (subdomain solves),
// Step 3 (CG on the interface with the BDDC preconditioner of Algorithm 2)
// and the post-correction.  Phases are separated by a grid barrier.  Per
// subdomain work units are processed by one warp each (global warps take
// contiguous chunks of units); coarse work units are blocks of coarse rows
// processed by one CTA each.
//
// Conventions of the packed data are those of bddc_internal.hpp: every
// per-subdomain operator is stored input-major (entry (out, in) at
// [in * n_out + out]) so that the lane computing one output reads
// consecutive addresses together with its neighbours; the restriction
// Psi^T r is a warp dot product over a contiguous row of PsiT.
//
// Two precisions: FP64 everywhere (S, F, Psi, coarse inverse), or the mixed
// path: F and Psi in FP32, and S and the coarse inverse stored as FP32 pairs
// (hi + lo, 48 significant bits) applied with compensated FP32 arithmetic,
// since FP64 arithmetic on GB300 runs at about 1/64 of the FP32 rate.  The
// mixed path keeps the preconditioner symmetric and its output exactly
// balanced, and ends with an FP64 coarse pressure correction.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bddc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCoarseRows = 16;             // coarse rows per work unit (default; Params::coarse_rows)
constexpr int64_t kDiropPartCost = 32768;    // largest n_out x n_Gamma of one operator-apply unit
constexpr long long kBarrierWaitNs = 10000000000LL;  // a grid-barrier wait past 10 s is an error
constexpr int kActMaxInst = 4096;           // largest batch whose CG phases are rebalanced over active instances

// A unit of the sparse coarse solve's sweeps (built on the host): node v,
// block blk of 32 outputs (boundary rows of H^T t in the forward sweep, pivot
// rows of x in the backward sweep) and the chunk [k0, k1) of its dot
// products (pivots forward; the concatenated columns [P, B] backward), with
// every offset the unit reads, so that one 64-byte record (four 16-byte
// loads) starts it.  The offsets are 32-bit: the setup rejects a factor or
// a coarse system past 2^31 entries for the sparse solver.
struct __align__(16) CsUnit {
    int blk, k0, k1, b;    // output block, chunk, instance
    int pp, q, nch, ich;   // the node's pivots and boundary, chunks of the block, this chunk
    int od;                // front dofs of the node (cn_idx)
    int om;                // the chunk's matrix: H (forward) or X (backward)
    int ou;                // the node's update vector in cs_u (forward) or H^T (backward)
    int cs;                // the instance's coarse system vectors
    int pof, cof;          // the block's partial sums and arrival counter
    int pad0, pad1;
};
constexpr int kCsChunk = 32;  // terms of a unit's dot products
constexpr int kCsMaxLevels = 62;  // tree depths whose unit offsets are staged in shared memory

struct GridSync {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};

// per-instance CG state (written by the warp that owns the instance)
struct InstState {
    int done;        // 1 once the instance left the CG loop
    int status;      // BDDC_OK / BDDC_E_NOT_CONVERGED / BDDC_E_BREAKDOWN
    int iterations;
    int fin;         // 1 + the CG phase (phase_index) in which it left the loop; 0 while active
    double r0, floor, rho0, relres;
};

// Index of a CG phase, for the active-instance snapshots: the PROLONG that
// decides iteration k (its convergence test) is 4k, the DIROP, UPDATE and
// COARSE of iteration k are 4k + 1, 4k + 2, 4k + 3.  An instance whose fin
// is 0 or above P is active in phase P: a warp reading fin during the phase
// in which it is written sees either 0 or P + 1, both "active", so all warps
// of a phase agree.
__host__ __device__ constexpr int phase_index(int k, int kind) { return 4 * k + kind; }
enum : int { kPhProlong = 0, kPhDirop = 1, kPhUpdate = 2, kPhCoarse = 3 };

struct Params {
    // instances
    int n_inst;
    const int64_t *inst_goff, *inst_ng, *inst_coff, *inst_ncn, *inst_ncf, *inst_kinv_off, *inst_s0, *inst_s1;
    const int64_t* inst_cfoff;  // prefix offsets of the coarse flux dofs
    const double* inst_vol;
    // subdomains
    int64_t n_sub;
    const int64_t* warp_sub0;  // per warp of the solve launch: first subdomain of its range (warps + 1)
    // operator-apply units: a subdomain whose S^i block exceeds kDiropPartCost
    // entries is applied in parts, each a range of its outputs (dunit[u]:
    // subdomain, (first output << 16) | end output), so that no part is
    // longer than a warp's share of the phase; units of a subdomain are
    // consecutive, sub_du0 (n_sub + 1) and inst_du0 (n_inst + 1) their first
    const int2* dunit;
    const int64_t *sub_du0, *inst_du0;
    const int64_t* warp_du0;  // per warp: first unit of its range (warps + 1)
    int64_t n_du;
    const int *sub_inst, *sub_ng, *sub_ni, *sub_nc, *sub_m, *sub_local;
    const int64_t *off_S, *off_F, *off_P, *off_Gpre, *off_Gpost, *off_slot, *off_cslot, *off_cell, *off_int;
    const double* sub_d;
    const int *slot_g, *slot_partner;
    const double *slot_w, *slot_dsig;
    const int* cslot_c;
    const int *slot_fcs, *cslot_n;   // net-flux row of each slot; dofs per net-flux row
    const double* slot_coef;
    const int *slot_fperm, *cslot_fstart;  // slots grouped by net-flux row
    const double* slot_fcoefp;             // their coefficients, same order
    // mixed path: weights, d*sigma and 1/n as FP32 pairs; coefficients as FP32
    const float2 *slot_w2, *slot_dsig2, *cslot_inv2;
    const float *slot_coef_f, *slot_fcoefp_f;
    const int64_t *cell_gid, *int_fid, *g_fid;
    const double* g_bsign;
    const int *c_slot_a, *c_slot_b;
    // full-space form of the operator (BDDC_FORM_FULL): per slot the RT0 mass
    // coefficient of its face in its cell, the cell's other face along the
    // axis and the cell with the face's side (see the setup's Packed)
    const double* slot_fk;
    const int *slot_fopp, *slot_fcell;
    // coarse units (inst_cu0: first unit of each instance, n_inst + 1 entries)
    // of coarse_rows rows each
    int64_t n_cunits;
    int coarse_rows;
    const int *cunit_inst, *cunit_row0;
    const int64_t* inst_cu0;
    // active-instance snapshots (per CTA, in shared memory): 0 = off (one
    // instance, or more than kActMaxInst), else n_inst
    int act_n;
    // matrices: S and Kinv are double (FP64 path) or float2 pairs (mixed);
    // F and P are double or float; P64 is always FP64
    const void *S, *F, *P, *Kinv;
    const double *P64, *Gpre, *Gpost;
    const float2* Gpost2;  // mixed path: Gpost as FP32 pairs
    // work vectors
    double *x, *rbuf0, *rbuf1, *dbuf0, *dbuf1, *g, *u0;        // interface
    double *ql, *zl, *yl, *rl, *tl;                            // local slots
    double* rcl;                                               // coarse slots
    double* wc;                                                // coarse vectors
    double *xp, *dp0, *dp1, *zp, *prhs;                        // per subdomain
    double *part_dq, *part_rr, *part_rz, *part_a1, *part_a2;   // per subdomain partials (part_dq: per operator-apply unit)
    int* inst_cnt;      // per instance and partial kind: arrivals of subdomain partials
    double* inst_tot;   // per instance: totals of the partials (rr, rz, dq, a1, a2)
    InstState* st;
    double *alpha_hist, *beta_hist, *rho_hist;                 // n_inst x (maxit + 1)
    int* n_active;
    GridSync* gsync;
    // sparse coarse solver (coarse_sparse = 1, bddc_coarse.cpp): the
    // multifrontal factor of every instance's coarse problem, per node X
    // (p x p, symmetric), H (p x q) and H^T (q x p); per front position its
    // dof and the children's update entries (cn_idx); the coarse system
    // vectors (right-hand side b, forward values t, solution x, the nodes'
    // update vectors u); the sweep units per tree depth (fw_off, bw_off:
    // prefix offsets) with their partial sums and arrival counters
    int coarse_sparse, cn_levels;
    const int64_t* inst_csoff;
    const double *cn_X, *cn_H, *cn_HT;
    double *cs_b, *cs_t, *cs_x, *cs_u;
    const int64_t *fw_off, *bw_off;
    const CsUnit *fw_unit, *bw_unit;
    const int4* cn_idx;  // per front position: (instance-local dof, children's update indices c0, c1, -)
    int *cs_fcnt, *cs_bcnt;
    double *cs_fpart, *cs_bpart;
    // phase timestamps (CTA 0 at each barrier): pairs (phase id, ns)
    long long* tstamp;
    int tstamp_cap;
    // io
    const double *f_in, *bc_in;
    double *flux_out, *p_out;
    // the full-space system (true residual of the solution): per instance
    // dim, nx, ny, nz, the cell size, face and cell offsets; per cell 1/k per
    // axis (stride 3); per face its boundary type (-1 inside, 0 no flow, 1
    // pressure); per (instance, chunk) CTA four partial sums
    const int* inst_grid;
    const double *inst_h, *cell_kinv;
    const int64_t *inst_face_off, *inst_cell_off;
    const int8_t* face_bct;
    double *tr_part, *tr_out;
    // control
    int maxit;
    double tol;
    int max_ng, max_in_post, max_ncn, max_m;
    int max_ext;  // per-warp extension area (full form: max n_I + n_cells; else 0)
};

}  // namespace bddc

// Device-side data layout and phase functions of the BDDC solve.
//
// One persistent cooperative kernel runs Algorithm 1 of the paper for every
// instance of a batch: Step 1 (coarse solve), Step 2 (subdomain solves),
// Step 3 (CG on the interface with the BDDC preconditioner of Algorithm 2)
// and the post-correction.  Phases are separated by a grid barrier; work
// units are subdomains (or blocks of coarse rows) assigned to CTAs in
// contiguous chunks.
//
// Conventions of the packed data are those of bddc_internal.hpp: every
// per-subdomain operator is stored input-major (entry (out, in) at
// [in * n_out + out]) so that the thread computing one output reads
// consecutive addresses together with its neighbours; the restriction
// Psi^T r is a warp dot product over a contiguous row of PsiT.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bddc {

constexpr int kThreads = 128;
constexpr int kCoarseRows = 8;              // coarse rows per work unit
constexpr long long kSpinLimit = 1LL << 24; // grid-barrier spins before giving up

struct GridSync {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};

// per-instance CG state (written by the instance's owner CTA)
struct InstState {
    int done;        // 1 once the instance left the CG loop
    int status;      // BDDC_OK / BDDC_E_NOT_CONVERGED / BDDC_E_BREAKDOWN
    int iterations;
    int pad;
    double r0, floor, rho0, relres;
};

struct Params {
    // instances
    int n_inst;
    const int64_t *inst_goff, *inst_ng, *inst_coff, *inst_ncn, *inst_ncf, *inst_kinv_off, *inst_s0, *inst_s1;
    const int64_t* inst_cfoff;  // prefix offsets of the coarse flux dofs
    const double* inst_vol;
    // subdomains
    int64_t n_sub;
    const int *sub_inst, *sub_ng, *sub_ni, *sub_nc, *sub_m, *sub_local;
    const int64_t *off_S, *off_F, *off_P, *off_Gpre, *off_Gpost, *off_slot, *off_cslot, *off_cell, *off_int;
    const double* sub_d;
    const int *slot_g, *slot_partner;
    const double *slot_w, *slot_dsig;
    const int* cslot_c;
    const int64_t *cell_gid, *int_fid, *g_fid;
    const double* g_bsign;
    const int *c_slot_a, *c_slot_b;
    // coarse units
    int64_t n_cunits;
    const int *cunit_inst, *cunit_row0;
    // matrices
    const double *S, *Gpre, *Gpost, *Kinv;
    const void *F, *P;
    // work vectors
    double *x, *rbuf0, *rbuf1, *dbuf0, *dbuf1, *g, *u0;        // interface
    double *ql, *zl, *yl, *rl, *tl;                            // local slots
    double* rcl;                                               // coarse slots
    double* wc;                                                // coarse vectors
    double *xp, *dp0, *dp1, *zp, *prhs;                        // per subdomain
    double *part_dq, *part_rr, *part_rz, *part_a1, *part_a2;   // per subdomain partials
    InstState* st;
    double *alpha_hist, *beta_hist, *rho_hist;                 // n_inst x (maxit + 1)
    int* n_active;
    GridSync* gsync;
    // io
    const double *f_in, *bc_in;
    double *flux_out, *p_out;
    // control
    int maxit;
    double tol;
    int max_ng, max_in_post, max_ncn;
};

}  // namespace bddc

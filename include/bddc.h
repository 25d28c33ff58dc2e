/*
 * bddc.h - C ABI of the GB300 adaptive BDDC solver for mixed RT0/P0 Darcy flow.
 *
 * Method: B. Sousedik, "On adaptive BDDC for the flow in heterogeneous porous
 * media" (arXiv:1901.02090).  The library solves the saddle-point system of
 * Sec. 4, eq. (system),
 *     [A  B^T] [u]   [g]
 *     [B  0  ] [p] = [f],
 * with a(u,v) = int k^{-1} u.v, b(u,q) = -int (div u) q, <f,q> = -int f q
 * (Sec. 2, eqs. (a), (b), (rhs)), lowest-order Raviart-Thomas fluxes and
 * piecewise-constant pressures on a Cartesian grid, by Algorithm 1 of the
 * paper: a coarse solve (Step 1), independent subdomain solves (Step 2), and
 * conjugate gradients on the divergence-free correction preconditioned by
 * BDDC (Step 3, Algorithm 2), with flux constraints selected by Algorithm 3.
 *
 * Data conventions (all arrays are in the caller's memory, host or device;
 * the library detects which with cudaPointerGetAttributes and copies them):
 *   - cells are numbered c = i + nx*(j + ny*k);
 *   - faces are numbered axis-major (all x-faces, then y, then z); inside an
 *     axis a face is numbered lexicographically over the grid extended by
 *     one along that axis;
 *   - a flux is the total normal flux through a face, positive along +axis;
 *   - pressure is one value per cell;
 *   - f is the source density per unit volume (positive = injection);
 *   - bc_type has one entry per face: -1 inside the domain, 0 no-flow
 *     boundary (zero normal flux), 1 prescribed pressure (value in
 *     bc_value at solve time).  In 2D the grid has nz = 1 and unit thickness.
 *   - a batch of instances is solved together: per-instance arrays are
 *     concatenated in instance order.
 *
 * Errors: every function returns BDDC_OK (0) or a negative code; the text
 * of the last error of a handle is returned by bddc_last_error.  No function
 * aborts the process or faults the GPU on invalid input.
 *
 * Threading: a handle is used by one host thread at a time; all its GPU work
 * is ordered on the stream given at setup.
 */
#ifndef BDDC_H
#define BDDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BDDC_OK 0
#define BDDC_E_INVALID_ARG (-1)   /* bad size, pointer or option */
#define BDDC_E_PARTITION (-2)     /* empty or face-disconnected subdomain, bad ids */
#define BDDC_E_PERM (-3)          /* permeability not finite or not positive */
#define BDDC_E_OOM (-4)           /* device or host allocation failed */
#define BDDC_E_NOT_CONVERGED (-5) /* maxit reached; outputs hold the last iterate */
#define BDDC_E_BREAKDOWN (-6)     /* (r,z) <= 0 or (d,Kd) <= 0 in CG */
#define BDDC_E_TIMEOUT (-7)       /* a device-side wait exceeded its limit */
#define BDDC_E_CUDA (-8)          /* a CUDA runtime call failed */
#define BDDC_E_SETUP (-9)         /* a local or coarse factorisation failed */

/* Precision of the subdomain-correction operators (Algorithm 2, step 2) and
 * of the coarse basis: FP64, or FP32 storage with FP32 arithmetic.  The
 * operator, the CG recurrence, the inner products and the coarse solve are
 * always FP64. */
#define BDDC_PREC_FP64 0
#define BDDC_PREC_FP32 1

/* Weights of the averaging operator E (Sec. 3), one value per side of each
 * face Gamma^{ij} (1 on pressure faces): multiplicity 1/2; stiffness the
 * face's share of the diagonals of the local a-form matrices,
 * sum_F A^i_ee / sum_F (A^i_ee + A^j_ee), which for RT0 is the rho-scaling
 * k_i^-1 / (k_i^-1 + k_j^-1) when k jumps across subdomain interfaces only
 * (Sec. 5).  The weights are constant along each face because the net-flux
 * constraints keep the Step-2 flux conservative only then (Sec. 3, Remark
 * "scaling"). */
#define BDDC_SCALING_MULTIPLICITY 0
#define BDDC_SCALING_STIFFNESS 1

/* Constraint set: the flux coarse dofs of each face Gamma^{ij} between two
 * subdomains (Sec. 3.1, eq. (C^i)).  All modes start from the initial
 * net-flux constraint of every face (Assumption 1) and add rows per face,
 * orthonormalised against the face's rows (a row in their span adds
 * nothing):
 *   ADAPTIVE  the rows of Algorithm 3 when tau > 0 (the method; tau <= 0:
 *             the initial constraints alone);
 *   MSMFEM    one row per face, the comparison method of Sec. 5: the flux on
 *             the face dofs of the local Darcy problem on the face's pair of
 *             subdomains with the sources 1/|Omega^i| on Omega^i and
 *             -1/|Omega^j| on Omega^j and no flow through the pair's
 *             boundary (the setup has no sources, so the uniform
 *             distribution is used in every subdomain; well-weighted rows
 *             can be given as EXPLICIT rows); tau is ignored;
 *   EXPLICIT  the caller's rows (bddc_instance.n_rows ...); tau is ignored.
 * bddc_stats.n_adaptive counts the rows added by any mode; omega_tilde is
 * the indicator of the constraints Algorithm 3 ended with (of the initial
 * constraints in the MSMFEM and EXPLICIT modes). */
#define BDDC_CONSTRAINTS_ADAPTIVE 0
#define BDDC_CONSTRAINTS_MSMFEM 1
#define BDDC_CONSTRAINTS_EXPLICIT 2

/* Coarse solver (Algorithm 1, the coarse problem of Step 1 and of every
 * preconditioner application).  Dense: the inverse of the coarse matrix,
 * applied as one dense matrix-vector product (per instance n_c^2 doubles).
 * Sparse: a multifrontal factorisation over a nested dissection of the
 * subdomains, applied by forward and backward sweeps over the dissection
 * tree.  Auto: dense while every instance has at most
 * BDDC_COARSE_DENSE_MAX coarse dofs, sparse otherwise. */
#define BDDC_COARSE_AUTO 0
#define BDDC_COARSE_DENSE 1
#define BDDC_COARSE_SPARSE 2
#define BDDC_COARSE_DENSE_MAX 2048

/* Form of the Step-3 operator (CG of Algorithm 1 on the divergence-free flux
 * correction; both forms give the same iterates in exact arithmetic).
 * Condensed: the interface problem of Sec. 3 (interiors eliminated by
 * static condensation); each subdomain applies its flux Schur complement
 * S^i as a dense n_Gamma^2 block.  Full: the iterates live in the full
 * RT0/P0 space as discrete-harmonic extensions of their interface values.
 * Each iteration extends the direction into the subdomain interiors
 * (interior fluxes and cell pressures, the interface columns of the
 * post-correction map, plus the subdomain's pressure constant) and applies
 * the mixed operator of Sec. 2 to it matrix-free, face by face; its rows on
 * the interior faces and cells vanish by construction, and its interface
 * rows are S^i applied to the direction.  The full form reads
 * n_Gamma x (n_I + n_cells) extension entries per subdomain instead of
 * n_Gamma^2 and requires BDDC_PREC_FP64. */
#define BDDC_FORM_CONDENSED 0
#define BDDC_FORM_FULL 1

typedef struct {
    int dim;      /* 2 or 3 */
    int n[3];     /* cells per axis; n[2] == 1 in 2D */
    double h[3];  /* cell size per axis; h[2] == 1 in 2D */
} bddc_grid;

typedef struct {
    bddc_grid grid;
    const double* perm;       /* n_cells * perm_ncomp, > 0; k per cell (isotropic)
                                 or per cell and axis (diagonal tensor) */
    int perm_ncomp;           /* 1 or dim */
    const int32_t* partition; /* n_cells subdomain ids 0..N-1 (boxes or any
                                 face-connected sets) */
    const int8_t* bc_type;    /* n_faces, see above */
    /* BDDC_CONSTRAINTS_EXPLICIT only (else 0 / NULL): n_rows constraint rows;
       row r has the faces row_face[row_ptr[r] .. row_ptr[r + 1]) (face ids of
       this instance) with the coefficients row_coef[same range].  All faces
       of a row must be interface dofs of one face Gamma^{ij} between two
       subdomains; otherwise the setup fails with BDDC_E_INVALID_ARG. */
    int n_rows;
    const int64_t* row_ptr;   /* n_rows + 1, row_ptr[0] = 0, non-decreasing */
    const int64_t* row_face;
    const double* row_coef;
} bddc_instance;

typedef struct {
    /* Algorithm 3 threshold tau: adaptive flux constraints are added on every
     * face where the local eigenproblem (Sec. 3.1, eq.
     * (eigenvalue-problem-local-matrix)) has eigenvalues above tau.
     * tau <= 0 or infinite: face-average constraints only (Assumption 1). */
    double tau;
    int scaling;          /* BDDC_SCALING_*, weights of E (Sec. 3, Remark) */
    int precision;        /* BDDC_PREC_* */
    int maxit;            /* CG iteration limit (> 0) */
    int pressure_scaling; /* 1: rescale the pressure block by D (Sec. 4) */
    int n_threads;        /* host threads used by setup; 0 = all cores */
    int coarse_solver;    /* BDDC_COARSE_* */
    int formulation;      /* BDDC_FORM_*; BDDC_FORM_FULL needs BDDC_PREC_FP64 */
    int constraints;      /* BDDC_CONSTRAINTS_* */
    int autotune;         /* 1: pick the launch's work layout by timing short probe solves at
                             setup (see bddc_get_tuning); 0: the fixed heuristic */
} bddc_options;

typedef struct {
    int iterations;        /* CG iterations of Step 3 */
    int status;            /* BDDC_OK, BDDC_E_NOT_CONVERGED or BDDC_E_BREAKDOWN */
    double kappa;          /* Lanczos estimate from the CG coefficients (Sec. 5); computed on the
                              first bddc_get_stats call after a solve */
    double relres;         /* final ||r||/||r_0|| of the reduced system */
    double omega_tilde;    /* condition indicator, eq. (indicator); 0 if none */
    int n_subdomains;      /* N */
    int n_interface;       /* interface flux dofs (incl. pressure faces) */
    int n_coarse;          /* coarse dofs: flux constraints + N pressures */
    int n_adaptive;        /* constraint rows added to the initial ones (Algorithm 3, MsMFEM or
                              the caller's rows, per bddc_options.constraints) */
    double true_relres;    /* ||r|| / ||rhs|| of the full RT0/P0 saddle system (Sec. 2) at the
                              returned flux and pressure: both block rows, every free face and
                              cell, applied matrix-free on the GPU after the solve */
} bddc_stats;

typedef struct bddc_handle bddc_handle;

/* Default options: tau = 0 (face averages), multiplicity scaling, FP64,
 * maxit = 5000, pressure scaling on, all host threads, automatic coarse
 * solver, condensed operator, adaptive constraint mode. */
void bddc_default_options(bddc_options* opt);

/* Set up one or more independent instances (Algorithm 1 setup: local
 * matrices (Sec. 2), constraints (Sec. 4.1 eq. (C^i), Algorithm 3), local
 * Schur complements and subdomain-correction operators (Algorithm 2), coarse
 * basis and coarse problem).  Inputs are copied; nothing is retained.
 * `cuda_stream` (a cudaStream_t, or NULL for the default stream) orders all
 * later GPU work of the handle.  On success *out receives a handle that owns
 * all device memory; on failure *out is NULL and the code says why. */
int bddc_setup(int n_instances, const bddc_instance* inst, const bddc_options* opt,
               void* cuda_stream, bddc_handle** out);

/* Solve all instances of the handle (Algorithm 1: Steps 1, 2 and 3 with the
 * BDDC preconditioner of Algorithm 2) to relative residual tol of the
 * reduced Step-3 system.
 *   f         : sum n_cells, source density per cell
 *   bc_value  : sum n_faces, pressure on bc_type == 1 faces (others ignored)
 *   flux      : sum n_faces (out), normal flux per face (0 on no-flow faces)
 *   pressure  : sum n_cells (out)
 *   iterations: n_instances (out, may be NULL)
 * Host or device pointers.  Returns BDDC_OK if every instance converged,
 * else the first failing instance's code (outputs still written). */
int bddc_solve(bddc_handle* h, const double* f, const double* bc_value, double tol,
               double* flux, double* pressure, int* iterations);

/* Per-instance statistics of the last solve. */
int bddc_get_stats(const bddc_handle* h, int instance, bddc_stats* out);

/* Sizes of the handle: instances, total interface dofs (the length of the
 * vectors of bddc_apply_operator), total subdomains. */
int bddc_sizes(const bddc_handle* h, int* n_instances, int64_t* n_interface,
               int64_t* n_subdomains);

/* The Step-3 reduced operator (Sec. 3, eqs. (corr-reduced-1/2)) on device
 * vectors: q = S u + B_0^T p0 with S = sum_i R_i^T S^i R_i, where u has
 * n_interface entries (interface flux dofs of all instances, each
 * instance's dofs sorted by global face id) and p0 one entry per subdomain
 * (subdomain pressure constants in the rescaled variables of Sec. 4).
 * Device pointers only; ordered on the handle's stream. */
int bddc_apply_operator(bddc_handle* h, const double* u, const double* p0, double* q);

/* The BDDC preconditioner (Algorithm 2) on device vectors: residual r
 * (n_interface) -> (z, z0), z the averaged flux correction (n_interface),
 * z0 the coarse pressure per subdomain. */
int bddc_apply_preconditioner(bddc_handle* h, const double* r, double* z, double* z0);

/* Subassembled operator apply from caller-owned device data, the kernel of
 * eqs. (corr-reduced-1/2) without a handle: q = sum_i R_i^T S^i R_i u.
 *   n_sub       : number of subdomains
 *   ng          : n_sub local interface sizes (each 0..1024)
 *   slot_offset : n_sub + 1 prefix offsets of the local slots: slot_offset[0]
 *                 = 0 and slot_offset[s + 1] - slot_offset[s] = ng[s]
 *   S_offset    : n_sub offsets (in doubles) of each S^i in S
 *   S           : the dense symmetric S^i, row-major, ng x ng each
 *   gidx        : slot -> global interface index (0..n_interface-1)
 *   partner     : slot -> slot of the other copy of the same dof, or -1
 *   u           : n_interface input
 *   q           : n_interface output (every entry with a slot is written)
 *   slot_scratch: caller-owned scratch of slot_offset[n_sub] doubles
 * Device pointers; stream is a cudaStream_t or NULL.  ng and slot_offset are
 * read back on `stream` (the call waits for the work queued there before
 * it) and checked on the host: sizes outside 0..1024 or offsets that are not
 * the prefix sums of ng give BDDC_E_INVALID_ARG before any launch (message
 * from bddc_last_error(NULL)).  The kernels skip any slot, partner or
 * interface index outside its buffer, so bad index tables give wrong values
 * but no access outside u, q and the scratch. */
int bddc_subassembled_apply(int n_sub, const int* ng, const int64_t* slot_offset,
                            const int64_t* S_offset, const double* S, const int* gidx,
                            const int* partner, int64_t n_interface, const double* u,
                            double* q, double* slot_scratch, void* stream);

/* Allocation-free variant of bddc_subassembled_apply (the paper has no
 * counterpart: this is a library-integration entry point).  Some callers
 * cannot call cudaMalloc: code running where the device allocator is
 * forbidden or already reserved (inside a caller's memory pool or arena
 * that owns all device memory, in real-time or safety-certified loops that
 * allow no device allocation after start-up).  This entry point takes the
 * same inputs and output but no scratch argument: its per-slot scratch is a
 * fixed array in the library's device memory, BDDC_NOALLOC_MAX_SLOTS doubles
 * (4 MiB), held by every GPU that loads the library until the process
 * exits.  It makes no device allocation: no cudaMalloc, cudaFree or
 * allocating library routine (its host-side checks use small host buffers).
 *   - ng and slot_offset are read back on `stream` and checked as for
 *     bddc_subassembled_apply; slot_offset[n_sub] larger than
 *     BDDC_NOALLOC_MAX_SLOTS is rejected with BDDC_E_INVALID_ARG (message
 *     from bddc_last_error(NULL)); the kernels never address the array past
 *     slot_offset[n_sub], whatever the index tables hold;
 *   - the read-back synchronises `stream` before the kernels are queued;
 *   - the first call on a device looks up the array's device address on the
 *     current device (once per device); make that first call before any
 *     stream capture;
 *   - every call on a device shares the one array; it needs no clearing
 *     (each call writes every slot it reads), and calls whose kernels
 *     overlap on the GPU (different streams, or another host thread) race on
 *     it: order them on one stream or serialise them.
 * Device pointers; stream is a cudaStream_t or NULL. */
#define BDDC_NOALLOC_MAX_SLOTS (1 << 19)
int bddc_subassembled_apply_noalloc(int n_sub, const int* ng, const int64_t* slot_offset,
                                    const int64_t* S_offset, const double* S, const int* gidx,
                                    const int* partner, int64_t n_interface, const double* u,
                                    double* q, void* stream);

/* Work layout of the persistent solve kernel and how it was chosen.  Each
 * warp takes a contiguous range of subdomains of equal summed cost
 * n_Gamma^2 + balance_weight (the operator blocks plus a fixed latency per
 * subdomain); each CTA takes units of coarse_rows rows of the dense coarse
 * inverse.  With bddc_options.autotune the setup times the persistent kernel
 * itself on the handle's operators for every candidate: the weights 4096
 * (the heuristic), 0, 1024, 16384 and 65536, crossed, for the dense coarse
 * solver, with the unit sizes 16, 8 and 32 rows (those that leave the launch
 * grid unchanged).  A candidate is timed by probe launches of 2 and 8 CG
 * iterations on a constant right-hand side, in two round-robin rounds after
 * three warm-up launches, the minimum per candidate and length; the
 * candidates are compared by the predicted time of a 30-iteration solve
 * (the 2-iteration time plus 28 times the cost per iteration), and the
 * heuristic wins ties within 2 %.  The choice is cached per signature
 * (launch grid, batch size, interface and constraint sizes of every
 * subdomain, coarse sizes, precision, form) for later setups of the process.
 * A probe that fails to launch or times out leaves the heuristic in place.
 * Without autotune: 4096 and 16.  Tuning allocates the host-array staging
 * buffers of bddc_solve at setup.  Returns BDDC_OK, or BDDC_E_INVALID_ARG
 * for a null argument. */
typedef struct {
    int tuned;                /* 1: chosen by probe solves (or taken from the cache), 0: heuristic */
    int from_cache;           /* 1: the choice of an earlier setup with the same signature */
    double balance_weight;    /* C of the warp ranges */
    int coarse_rows;          /* rows of a dense-coarse work unit */
    double probe_ms;          /* the chosen layout's predicted 30-iteration solve time (0 if not tuned) */
    double probe_ms_default;  /* the heuristic layout's predicted time (0 if not tuned) */
} bddc_tuning;
int bddc_get_tuning(const bddc_handle* h, bddc_tuning* out);

/* Device time (ms) of the last solve's main kernel (the persistent Step 1-3
 * kernel), measured with CUDA events around its launch, and the algorithmic
 * bytes it moved (matrix entries and vectors per iteration times the
 * iterations, plus the pre- and post-processing passes). */
int bddc_last_solve_timing(const bddc_handle* h, double* kernel_ms, double* algorithmic_bytes);

/* Host-only inspection of the setup (no GPU needed): runs the same setup as
 * bddc_setup and keeps the packed operators in host memory, so that tests
 * and diagnostics can read them.  Arrays are exported by name:
 *   int32 : sub_inst sub_ng sub_ni sub_nc sub_m sub_local slot_g
 *           slot_partner cslot_c c_slot_a c_slot_b g_slot_a g_slot_b
 *           slot_fcs cslot_n slot_fperm cslot_fstart
 *   int64 : inst_goff inst_ng inst_coff inst_ncn inst_ncf inst_kinv_off
 *           inst_s0 inst_s1 inst_face_off inst_nfaces inst_cell_off
 *           inst_ncells off_S off_F off_P off_Gpre off_Gpost off_slot
 *           off_cslot off_cell off_int cell_gid int_fid g_fid
 *   double: inst_vol inst_omega sub_d slot_w slot_dsig slot_coef slot_fcoefp g_bsign S F P Gpre
 *           Gpost Kinv P64  (F and P are FP64 copies of the operators the
 *           GPU applies, FP32-rounded for FP32 setups; P64 is the FP64 basis)
 *   sparse coarse factor (empty with the dense coarse solver):
 *   int32 : cn_inst cn_p cn_q cn_depth cn_dof cn_c0 cn_c1
 *   int64 : inst_csoff inst_node0 cn_off_dof cn_off_X cn_off_H cn_off_u
 *   double: cn_X cn_H cn_HT
 * bddc_host_setup_query gives the element count and size (0 count for an
 * unknown name); bddc_host_setup_copy copies the array into dst. */
typedef struct bddc_host_setup bddc_host_setup;
int bddc_host_setup_create(int n_instances, const bddc_instance* inst, const bddc_options* opt,
                           bddc_host_setup** out);
/* The same, with the dense part of the local maps (S, G_pre, G_post) computed
 * on the current CUDA device, as bddc_setup and the serving loop do; they
 * agree with the host computation to rounding.  BDDC_E_CUDA without a GPU. */
int bddc_host_setup_create_gpu(int n_instances, const bddc_instance* inst, const bddc_options* opt,
                               bddc_host_setup** out);
int bddc_host_setup_query(const bddc_host_setup* hs, const char* name, int64_t* count, int* elem_bytes);
int bddc_host_setup_copy(const bddc_host_setup* hs, const char* name, void* dst);
void bddc_host_setup_destroy(bddc_host_setup* hs);
/* x = K_c^{-1} rhs for one instance with the setup's coarse solver, on the
 * host: the dense inverse, or the forward and backward sweeps over the
 * packed multifrontal factor in the order the device runs them.  rhs and x
 * are host arrays of n_c + N doubles (flux coarse dofs, then the subdomain
 * pressures).  BDDC_E_INVALID_ARG for a null pointer or a bad instance. */
int bddc_host_setup_coarse_solve(const bddc_host_setup* hs, int instance, const double* rhs, double* x);

/* Diagnostic copy of a device work vector of the last solve into host
 * memory: "x" "r0" "r1" "d0" "d1" "g" "u0" (interface), "ql" "zl" "yl" "rl"
 * "tl" (local slots), "rcl" (coarse slots), "wc" (coarse vectors), "xp" "zp"
 * "prhs" "part_rr" "part_rz" "part_dq" (per subdomain), "alpha" "beta" (the
 * CG coefficients, maxit + 1 per instance, instance-major).  *count
 * receives the length; dst may be NULL to query it. */
int bddc_debug_vector(const bddc_handle* h, const char* name, double* dst, int64_t* count);

/* Diagnostic phase timeline of the last solve: pairs (phase id, global
 * timer in ns) recorded by CTA 0 as each grid-wide phase of the persistent
 * kernel ended (ids: 0 start, 1 Step-1 restriction, 2 Step-1 coarse solve,
 * 3 u_0, 4 Step-2 residual, 5 f* and first restriction, 6 coarse solve,
 * 7 prolongation, 8 direction update and operator, 9 CG update and
 * restriction, 10-13 closing pressure correction); unused pairs are zero.
 * *count receives the number of int64 entries; pairs may be NULL. */
int bddc_debug_phase_times(const bddc_handle* h, int64_t* pairs, int64_t* count);

/* Failure-detection diagnostic of the bounded grid-barrier wait: launches
 * n_ctas (2..1024) CTAs that enter one grid barrier except the last, which
 * never arrives; the others give up after limit_ns (0 < limit <= 60 s) and
 * set the error flag.  Returns BDDC_E_TIMEOUT when the wait ran out as
 * designed (the device context stays usable), BDDC_OK if it did not,
 * BDDC_E_INVALID_ARG or BDDC_E_CUDA.  The solve kernel's barriers use the
 * same wait with a 10 s limit. */
int bddc_debug_barrier_timeout(long long limit_ns, int n_ctas);

const char* bddc_last_error(const bddc_handle* h);
const char* bddc_error_string(int code);
void bddc_destroy(bddc_handle* h);

/* ---- serving: continuous batching of independent solves --------------------
 * Not a method of the paper: a request loop over the batch solver above, for
 * a stream of independent problems of any sizes.
 *
 * bddc_submit copies a request (host arrays) and returns a ticket at once.
 * Two setup threads take the requests in arrival order (consecutive requests
 * with equal tol, at most max_batch per batch), run their setup (Algorithm 3
 * and the local maps; the dense parts on the GPU), admit a batch when its
 * device footprint fits the HBM budget beside the batches already on the
 * device, and upload it.  A solve thread runs the admitted batches on the
 * GPU one after another (one launch of the persistent kernel each).  The
 * setups of two batches overlap each other (one on the host while the other
 * is on the GPU) and the solve of the current batch; requests that arrive
 * while batches are being set up or solved join a later batch.  Results are
 * collected by ticket with bddc_poll (and waited for with bddc_wait).
 *
 * The result of a request is bitwise the same as bddc_setup + bddc_solve of
 * that problem alone with the same options: the kernel's arithmetic for one
 * instance does not depend on the other instances of its batch.
 *
 * A request that fails (invalid input, setup failure, no convergence) reports
 * its own error code and does not fail the other requests of its batch.
 * All request and result arrays are host memory.  One host thread at a time
 * may call the functions of one server. */
#define BDDC_PENDING 1 /* bddc_poll / bddc_wait: the request is not done yet */

typedef struct bddc_server bddc_server;

typedef struct {
    double queue_ms;   /* submission -> the host setup of its batch starts */
    double setup_ms;   /* host setup + wait for HBM admission + upload of its batch */
    double solve_ms;   /* solve of its batch on the GPU, result copies included */
    double latency_ms; /* submission -> result available */
    int batch_size;    /* requests solved in the same launch, itself included */
    int64_t batch_id;
} bddc_request_info;

typedef struct {
    int64_t submitted, completed, failed, batches;
    size_t device_bytes_in_use, device_bytes_peak; /* of the batches set up or solving */
} bddc_server_info;

/* opt as for bddc_setup (NULL: defaults); hbm_budget_bytes > 0 bounds the
 * device memory of the batches on the device at a time (a batch larger than
 * the budget on its own fails its requests with BDDC_E_OOM); max_batch >= 1.
 * Uses the current CUDA device. */
int bddc_server_create(const bddc_options* opt, size_t hbm_budget_bytes, int max_batch, bddc_server** out);

/* inst: the problem (as for bddc_setup); f: n_cells sources; bc_value:
 * n_faces boundary values; tol > 0.  The arrays are copied before the call
 * returns.  *ticket identifies the request. */
int bddc_submit(bddc_server* s, const bddc_instance* inst, const double* f, const double* bc_value, double tol,
                uint64_t* ticket);

/* BDDC_PENDING if the request is not done; otherwise copies its results
 * (flux: n_faces, pressure: n_cells, iterations, stats, info; any may be
 * NULL), releases the ticket and returns the request's status: BDDC_OK or
 * its error code (BDDC_E_NOT_CONVERGED: the outputs hold the last iterate).
 * An unknown or released ticket: BDDC_E_INVALID_ARG. */
int bddc_poll(bddc_server* s, uint64_t ticket, double* flux, double* pressure, int* iterations, bddc_stats* stats,
              bddc_request_info* info);

/* Waits until the request is done (BDDC_OK) or timeout_s seconds passed
 * (BDDC_PENDING); timeout_s < 0 waits without limit. */
int bddc_wait(bddc_server* s, uint64_t ticket, double timeout_s);

int bddc_server_get_info(bddc_server* s, bddc_server_info* info);

/* Drops the requests not yet set up, lets the batches on the device finish,
 * stops the threads and frees everything. */
void bddc_server_destroy(bddc_server* s);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_H */

// Internal types shared by the host setup (bddc_setup.cpp) and the device
// code (bddc_kernels.cu).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/bddc.h"

namespace bddc {

// Host-side result of the setup of all instances, packed for upload.
// Every per-subdomain matrix is stored "input-major": entry (out, in) of an
// operator is at [in * n_out + out], so that a thread per output reads
// consecutive addresses when it walks the inputs.
struct Packed {
    // per instance
    std::vector<int64_t> inst_goff, inst_ng;        // interface vector offset, size
    std::vector<int64_t> inst_coff, inst_ncn;       // coarse vector offset, n_cf + N
    std::vector<int64_t> inst_ncf;                  // coarse flux dofs
    std::vector<int64_t> inst_kinv_off;             // offset of the coarse inverse
    std::vector<int64_t> inst_s0, inst_s1;          // subdomain range
    std::vector<int64_t> inst_face_off, inst_nfaces;
    std::vector<int64_t> inst_cell_off, inst_ncells;
    std::vector<double> inst_vol;
    std::vector<int> inst_nadapt;
    std::vector<double> inst_omega;
    // per subdomain
    std::vector<int> sub_inst, sub_ng, sub_ni, sub_nc, sub_m, sub_local;
    std::vector<int64_t> off_S, off_F, off_P, off_Gpre, off_Gpost;
    std::vector<int64_t> off_slot, off_cslot, off_cell, off_int;  // n_sub + 1
    std::vector<double> sub_d;
    // per local interface slot
    std::vector<int> slot_g, slot_partner;
    std::vector<double> slot_w, slot_dsig;
    // per local interface slot: the local coarse slot of its face's net-flux
    // row and the row's coefficient (+1/-1); per local coarse slot: the
    // number of face dofs of a net-flux row (0 for adaptive rows)
    std::vector<int> slot_fcs, cslot_n;
    std::vector<double> slot_coef;
    // per subdomain the local slots grouped by net-flux row (slot_fperm,
    // indexed from the subdomain's slot offset) and, per local coarse slot,
    // the start of its group (-1 for adaptive rows)
    std::vector<int> slot_fperm, cslot_fstart;
    std::vector<double> slot_fcoefp;  // coefficient of slot_fperm[q], in the same order
    // per local coarse slot: instance-local coarse index
    std::vector<int> cslot_c;
    // per local cell / interior flux: index into the batched output arrays
    std::vector<int64_t> cell_gid, int_fid;
    // per global interface dof
    std::vector<int64_t> g_fid;
    std::vector<int> g_slot_a, g_slot_b;
    std::vector<double> g_bsign;  // +1 pressure face on a min side, -1 max side, 0 otherwise
    // per coarse flux dof (batched): the <= 2 coarse slots that hold it
    std::vector<int> c_slot_a, c_slot_b;
    // sparse coarse factor (coarse_sparse = 1): per instance the offset of
    // its coarse system vectors (n_cf + N + pure entries, inst_csoff) and of
    // its nodes (inst_node0, n_inst + 1 entries); per node (batched): the
    // instance, p, q, depth, offsets of its front dofs (P then B,
    // instance-local) and of X (p x p), H (p x q) and HT (q x p); per front
    // position the batched index, in the update array u, of the children's
    // update for that dof (-1: none)
    int coarse_sparse = 0;
    std::vector<int64_t> inst_csoff, inst_node0;
    std::vector<int> cn_inst, cn_p, cn_q, cn_depth;
    std::vector<int64_t> cn_off_dof, cn_off_X, cn_off_H, cn_off_u;
    std::vector<int> cn_dof;
    std::vector<int> cn_c0, cn_c1;
    std::vector<double> cn_X, cn_H, cn_HT;
    int64_t n_csys = 0, n_cu = 0;
    int cn_max_depth = 0;
    // the full-space system of every instance, for the true residual of a
    // solution (the RT0/P0 saddle system of Sec. 2 applied matrix-free):
    // per instance dim, nx, ny, nz and the cell size; per cell 1/k per axis
    // (stride 3); per face its boundary type
    std::vector<int> inst_grid;
    std::vector<double> inst_h, cell_kinv;
    std::vector<int8_t> face_bct;
    // the full-space form of the Step-3 operator (BDDC_FORM_FULL only), per local
    // interface slot: the RT0 mass coefficient h_a^2 / (|K| k_a) of the
    // slot's face in the subdomain's cell K on it; K's other face along the
    // same axis as an index into the subdomain's local fluxes (slots, then
    // ng + interior face) or -1 (a no-flow face); K as local cell r + 1 when
    // the face is K's lower face, -(r + 1) when it is its upper face
    std::vector<double> slot_fk;
    std::vector<int> slot_fopp, slot_fcell;
    // matrices
    std::vector<double> S, F64, P64, Gpre, Gpost, Kinv;
    std::vector<float> F32, P32;
    int precision = BDDC_PREC_FP64;
    // G_post computed on the GPU stays there: a device array in the layout
    // of Gpost (which is then empty on the host), freed with its last owner
    std::shared_ptr<double> dev_Gpost;
    int64_t dev_Gpost_count = 0;
    int64_t n_sub = 0, n_gamma = 0, n_coarse_vec = 0;
    int max_ng = 0, max_m = 0, max_ncn = 0, max_out_post = 0, max_in_post = 0;
};

// steps of iterative refinement of the dense local maps (host and device
// alike, so that both compute the same maps)
constexpr int kLocalRefinements = 1;

// the option values every entry point accepts
inline bool options_valid(const bddc_options& o) {
    return o.maxit > 0 && (o.precision == BDDC_PREC_FP64 || o.precision == BDDC_PREC_FP32) &&
           (o.scaling == BDDC_SCALING_MULTIPLICITY || o.scaling == BDDC_SCALING_STIFFNESS) &&
           o.coarse_solver >= BDDC_COARSE_AUTO && o.coarse_solver <= BDDC_COARSE_SPARSE && (o.autotune == 0 || o.autotune == 1) &&
           o.constraints >= BDDC_CONSTRAINTS_ADAPTIVE && o.constraints <= BDDC_CONSTRAINTS_EXPLICIT &&
           (o.formulation == BDDC_FORM_CONDENSED ||
            (o.formulation == BDDC_FORM_FULL && o.precision == BDDC_PREC_FP64));
}

struct SetupResult {
    int code = BDDC_OK;
    std::string msg;
};

// The coarse problem in element form (one element per subdomain, over its
// coarse dofs) and its multifrontal factor (bddc_coarse.cpp).
struct CoarseElement {
    std::vector<int> dofs;  // instance-local coarse dofs
    std::vector<double> E;  // dofs.size()^2, row-major
    double c[3] = {0.0, 0.0, 0.0};  // centroid of the subdomain
};
struct CoarseFactor {
    int n = 0, root = -1, max_depth = 0;
    // per node of the dissection tree, children before parents
    std::vector<int> parent, child0, child1, depth;
    std::vector<std::vector<int>> piv, bnd;   // the node's dofs P and its boundary B (sorted)
    std::vector<std::vector<double>> X, H;    // X = F_PP^{-1} (p x p), H = X F_PB (p x q), row-major
};
// is_pressure[d]: d is a subdomain pressure (kept out of a node's pivots
// once per node, see bddc_coarse.cpp)
SetupResult factor_coarse(int n, const std::vector<CoarseElement>& el, const std::vector<char>& is_pressure,
                          int leaf_max, int nthreads, CoarseFactor& f);
// x = K^{-1} b with the factor (host; the device sweeps mirror it)
void coarse_factor_solve(const CoarseFactor& f, const double* b, double* x);

// Dense part of the local maps of a batch of subdomains (the interior saddle
// solves behind S^i, G_pre and G_post, with iterative refinement), for the
// device implementation in bddc_setup_gpu.cu.  Per-subdomain blocks are
// concatenated; o_* are prefix offsets with n_sub + 1 entries.
struct LocalMapsBatch {
    int n_sub = 0;
    // per subdomain
    std::vector<int> dim, ng, ni, nc;
    std::vector<double> vol, d;
    std::vector<int64_t> o_cell, o_ng, o_ni, o_ch;
    // per cell and axis (stride 3): local lower / upper face (-1 absent) and h_a^2/|c|/k_a
    std::vector<int> clo, chi;
    std::vector<double> cs;
    // per interface dof: its cell, axis and side (0 lower, 1 upper)
    std::vector<int> gcell, gaxis, gside;
    // per interior dof, in chain order: interior index and Thomas factors
    // (rdfac: reciprocals of the pivots); per chain (o_ch, n_chains + 1
    // entries per subdomain): start position
    std::vector<int> order, cstart;
    std::vector<double> rdfac, lfac, off;
    // outputs, in the layouts of the host setup
    std::vector<int64_t> o_S, o_Gpre, o_Gpost;
    std::vector<double> S, GpreT;
    std::shared_ptr<double> dev_GpostT;  // G_post of every subdomain, on the device (o_Gpost layout)
    std::vector<int> status;  // per subdomain: BDDC_OK or BDDC_E_SETUP
};

// The adaptive face eigenproblems of a batch on the GPU (bddc_eigen_gpu.cu).
// Subdomains (those with an adaptive face): the interface Schur complement
// S^i (n x n row-major) and the weights w; faces: the two subdomains (batch
// indices), f face dofs with their positions in either subdomain's
// interface and the net-flux coefficients.  Outputs per face: omega^{ij},
// the number k of rows above tau and the rows (k x f at o_rows, capacity
// f x f), before the orthonormalisation against the face's existing rows.
struct FaceEigenBatch {
    std::vector<int> n;
    std::vector<int64_t> o_S, o_w;
    std::vector<double> S, w;
    std::vector<int> fi, fj, ff;
    std::vector<int64_t> o_f, o_rows;  // per face, n_face + 1 entries
    std::vector<int> pi, pj;
    std::vector<double> coef;
    double tau = -1.0;
    std::vector<double> omega, rows;
    std::vector<int> nrows, face_status, sub_status;
};
using FaceEigenDevice = int (*)(FaceEigenBatch& batch, std::string& err);
int face_eigen_device(FaceEigenBatch& batch, std::string& err);

// host copy of a device array of doubles (for the host-side export)
bool device_to_host(const double* dev, int64_t n, double* host);
using LocalMapsDevice = int (*)(LocalMapsBatch& batch, std::string& err);

// computes a batch's dense local maps on the current CUDA device
int local_maps_device(LocalMapsBatch& batch, std::string& err);

// host setup of a batch; with a device hook the dense part of the local
// maps runs there
SetupResult build_all(int n_inst, const bddc_instance* inst, const bddc_options& opt, Packed& out,
                      LocalMapsDevice device = nullptr, FaceEigenDevice eig_device = nullptr);

// device part of bddc_setup (bddc_kernels.cu): uploads the host setup of a
// batch, sizes the persistent launch, and returns the handle
int setup_from_packed(int n_instances, const bddc_options& opt, void* cuda_stream, Packed&& packed,
                      bddc_handle** out);
// device memory held by a handle (bytes)
size_t handle_device_bytes(const bddc_handle* h);

}  // namespace bddc

// Host-side setup of the BDDC operators (native C++, multithreaded).
//
// For every subdomain i (Sec. 3) this builds, from the RT0/P0 cell matrices
// (Sec. 2, eqs. (a), (b)) and the rescaled divergence block d_i B^i (Sec. 4,
// eq. (system-scaled)):
//   * the Stokes-harmonic solution map of the local problem with the pressure
//     constraint C_Q^i (cell volumes):
//       [A_II  dB_I^T  0 ] [u_I]   [-A_IG u_G          ]
//       [dB_I  0       v ] [p  ] = [d <f,q> - dB_G u_G  ]
//       [0     v^T     0 ] [mu ]   [0                  ]
//     eliminated in the order interior fluxes (A_II is a set of independent
//     tridiagonal chains, one per grid line), then pressures (dense (n_c+1)
//     LU);
//   * S^i, the interface Schur complement (the energy of the Stokes-harmonic
//     extension), and the maps used by Steps 2 and the post-correction;
//   * the constraints C^i (eq. (C^i)): one net-flux row per face Gamma^{ij}
//     (Assumption 1) and per group of pressure faces, plus the adaptive rows
//     of Algorithm 3;
//   * the subdomain correction F_i = Z (Z^T S Z)^{-1} Z^T, Z spanning null C^i
//     (Algorithm 2 step 2 restricted to the interface), and the coarse basis
//     Psi_i = (I - F_i S_i) C^T (C C^T)^{-1} (unit coarse values, minimal
//     energy);
// and per instance the coarse saddle-point matrix over (W_Pi, Q_0) and its
// inverse (Algorithm 1 step 1, Algorithm 2 step 1).
//
// Algorithm 3 is evaluated in the face-reduced form: for a jump delta across
// Gamma^{ij} the smallest pair energy is delta^T (T_i + T_j)^{-1} delta with
// T = (S^{-1})_FF, and the energy of (I - E^{ij}) w is delta^T S_F delta with
// S_F = W_j S^i_FF W_j + W_i S^j_FF W_i; the nonzero eigenvalues of
// eq. (eigenvalue-problem-local-matrix) are those of S_F delta =
// lambda (T_i + T_j)^{-1} delta on the face-constraint null space, and the
// row of eq. (constraints) is S_F delta_l on the face dofs (both halves of
// c_l, in global orientation).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

#include "bddc_internal.hpp"
#include "bddc_trace.hpp"
#include "dense.hpp"

namespace bddc {
namespace {

constexpr double kMassDiag = 1.0 / 3.0;
constexpr double kMassOff = 1.0 / 6.0;

struct Geometry {
    int dim, nx, ny, nz;
    double h[3], vol;
    int64_t n_cells, n_faces, face_off[4];
    int64_t face_id(int a, int64_t i, int64_t j, int64_t k) const {
        int64_t ex = nx, ey = ny;
        if (a == 0) ex += 1;
        if (a == 1) ey += 1;
        return face_off[a] + i + ex * (j + ey * k);
    }
    int64_t cell_face(int64_t c, int a, int side) const {
        int64_t i = c % nx, j = (c / nx) % ny, k = c / ((int64_t)nx * ny);
        if (side) { if (a == 0) ++i; else if (a == 1) ++j; else ++k; }
        return face_id(a, i, j, k);
    }
    // cell below (side 0) or above (side 1) face f along its axis, or -1
    int64_t face_cell(int64_t f, int side, int* axis) const {
        int a = 0;
        while (a + 1 <= dim - 1 && f >= face_off[a + 1]) ++a;
        *axis = a;
        int64_t r = f - face_off[a];
        int64_t ex = nx + (a == 0), ey = ny + (a == 1);
        int64_t i = r % ex, j = (r / ex) % ey, k = r / (ex * ey);
        int64_t pos = (a == 0) ? i : (a == 1) ? j : k;
        int64_t ext = (a == 0) ? nx : (a == 1) ? ny : nz;
        if (side == 0) {
            if (pos == 0) return -1;
            if (a == 0) --i; else if (a == 1) --j; else --k;
        } else {
            if (pos == ext) return -1;
        }
        return i + (int64_t)nx * (j + (int64_t)ny * k);
    }
};

struct Sub {
    std::vector<int64_t> cells;     // sorted instance cell ids
    std::vector<int64_t> faces;     // interface (sorted) then interior (sorted)
    int ng = 0, ni = 0, nc = 0, m = 0;
    double d = 1.0;
    std::vector<int> gidx;          // interface slot -> instance interface index
    std::vector<double> w, sigma, diagA;
    // per (local cell, axis): local face index of lower/upper face (-1 absent)
    std::vector<int> clo, chi;
    std::vector<double> cs;         // h_a^2 / |c| / k_a
    std::vector<double> S, GpreT, GpostT, Lchol;
    std::vector<double> C, F, PsiT;
    std::vector<int> cid;
    std::vector<int> fcs;        // interface slot -> local row of its net-flux constraint
    std::vector<double> fcoef;   // coefficient of that row on the slot
    std::vector<int> rown;       // local row -> face dofs (net-flux rows), 0 otherwise
};

struct Face {
    bool dir;                       // group of pressure faces
    int i, j;                       // subdomains (j = -1 for pressure groups)
    std::vector<int> gidx;          // instance interface indices, sorted by face id
    std::vector<double> coef;       // net-flux row (+1: normal out of subdomain i)
    std::vector<std::vector<double>> rows;
    std::vector<int> cids;
};

struct Inst {
    Geometry geo;
    std::vector<double> kinv;       // n_cells * dim, 1/k
    std::vector<int> part;
    int N = 0;
    std::vector<int8_t> bct;
    std::vector<int64_t> gamma;     // sorted face ids of the interface
    std::vector<Sub> subs;
    std::vector<Face> faces;
    int n_cf = 0, n_adapt = 0;
    bool pure = false;
    std::vector<double> Kinv;       // (n_cf + N) square (dense coarse solver)
    CoarseFactor cf;                // multifrontal coarse factor (sparse coarse solver)
    double omega = 0.0;
    // caller constraint rows (BDDC_CONSTRAINTS_EXPLICIT): CSR over face ids
    std::vector<int64_t> xrow_ptr, xrow_face;
    std::vector<double> xrow_coef;
};

template <class F>
void parallel_for(int64_t n, int nthreads, F&& fn) {
    if (n <= 0) return;
    nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(nthreads, n));
    if (nthreads == 1) {
        for (int64_t i = 0; i < n; ++i) fn(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t)
        th.emplace_back([&] {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                fn(i);
            }
        });
    for (auto& t : th) t.join();
}

int lower_index(const std::vector<int64_t>& v, int64_t x, int base) {
    auto it = std::lower_bound(v.begin() + base, v.end(), x);
    if (it == v.end() || *it != x) return -1;
    return (int)(it - v.begin());
}

// ---- validation and topology ------------------------------------------------
SetupResult read_instance(const bddc_instance& in, Inst& I) {
    SetupResult res;
    const bddc_grid& g = in.grid;
    if (g.dim != 2 && g.dim != 3) return {BDDC_E_INVALID_ARG, "grid.dim must be 2 or 3"};
    for (int a = 0; a < 3; ++a)
        if (g.n[a] < 1 || !(g.h[a] > 0) || !std::isfinite(g.h[a]))
            return {BDDC_E_INVALID_ARG, "grid sizes must be >= 1 and cell sizes positive"};
    if (g.dim == 2 && g.n[2] != 1) return {BDDC_E_INVALID_ARG, "2D grids need n[2] == 1"};
    if (!in.perm || !in.partition || !in.bc_type) return {BDDC_E_INVALID_ARG, "null instance array"};
    if (in.perm_ncomp != 1 && in.perm_ncomp != g.dim)
        return {BDDC_E_INVALID_ARG, "perm_ncomp must be 1 or dim"};
    Geometry& G = I.geo;
    G.dim = g.dim; G.nx = g.n[0]; G.ny = g.n[1]; G.nz = g.n[2];
    for (int a = 0; a < 3; ++a) G.h[a] = g.h[a];
    G.vol = g.h[0] * g.h[1] * g.h[2];
    G.n_cells = (int64_t)G.nx * G.ny * G.nz;
    G.face_off[0] = 0;
    G.face_off[1] = (int64_t)(G.nx + 1) * G.ny * G.nz;
    G.face_off[2] = G.face_off[1] + (int64_t)G.nx * (G.ny + 1) * G.nz;
    G.face_off[3] = G.face_off[2] + (g.dim == 3 ? (int64_t)G.nx * G.ny * (G.nz + 1) : 0);
    G.n_faces = G.face_off[g.dim];
    if (G.n_cells > (int64_t)1 << 30) return {BDDC_E_INVALID_ARG, "grid too large"};
    I.kinv.resize((size_t)G.n_cells * g.dim);
    for (int64_t c = 0; c < G.n_cells; ++c)
        for (int a = 0; a < g.dim; ++a) {
            const double k = in.perm[c * in.perm_ncomp + (in.perm_ncomp == 1 ? 0 : a)];
            if (!(k > 0) || !std::isfinite(k)) return {BDDC_E_PERM, "permeability must be finite and > 0"};
            I.kinv[c * g.dim + a] = 1.0 / k;
        }
    I.part.assign(in.partition, in.partition + G.n_cells);
    int pmax = -1;
    for (int64_t c = 0; c < G.n_cells; ++c) {
        if (I.part[c] < 0) return {BDDC_E_PARTITION, "negative subdomain id"};
        pmax = std::max(pmax, I.part[c]);
    }
    I.N = pmax + 1;
    I.bct.assign(in.bc_type, in.bc_type + G.n_faces);
    bool any_dir = false;
    for (int64_t f = 0; f < G.n_faces; ++f) {
        int ax;
        const bool boundary = G.face_cell(f, 0, &ax) < 0 || G.face_cell(f, 1, &ax) < 0;
        const int t = I.bct[f];
        if (boundary ? (t != 0 && t != 1) : (t != -1))
            return {BDDC_E_INVALID_ARG, "bc_type must be -1 inside and 0 or 1 on the boundary"};
        any_dir |= (t == 1);
    }
    I.pure = !any_dir;
    if (in.n_rows < 0) return {BDDC_E_INVALID_ARG, "n_rows must be >= 0"};
    if (in.n_rows > 0) {
        if (!in.row_ptr || !in.row_face || !in.row_coef) return {BDDC_E_INVALID_ARG, "null constraint-row array"};
        I.xrow_ptr.assign(in.row_ptr, in.row_ptr + in.n_rows + 1);
        if (I.xrow_ptr[0] != 0) return {BDDC_E_INVALID_ARG, "row_ptr[0] must be 0"};
        for (int r = 0; r < in.n_rows; ++r)
            if (I.xrow_ptr[r + 1] < I.xrow_ptr[r]) return {BDDC_E_INVALID_ARG, "row_ptr must be non-decreasing"};
        const int64_t nnz = I.xrow_ptr[in.n_rows];
        I.xrow_face.assign(in.row_face, in.row_face + nnz);
        I.xrow_coef.assign(in.row_coef, in.row_coef + nnz);
        for (int64_t q = 0; q < nnz; ++q) {
            if (I.xrow_face[q] < 0 || I.xrow_face[q] >= G.n_faces) return {BDDC_E_INVALID_ARG, "row face id out of range"};
            if (!std::isfinite(I.xrow_coef[q])) return {BDDC_E_INVALID_ARG, "row coefficient not finite"};
        }
    }
    return res;
}

SetupResult build_topology(Inst& I) {
    Geometry& G = I.geo;
    const int dim = G.dim;
    std::vector<int64_t> count(I.N, 0);
    for (int p : I.part) count[p]++;
    for (int s = 0; s < I.N; ++s)
        if (count[s] == 0) return {BDDC_E_PARTITION, "subdomain ids must be 0..N-1 with none empty"};
    I.subs.assign(I.N, Sub());
    for (int64_t c = 0; c < G.n_cells; ++c) I.subs[I.part[c]].cells.push_back(c);
    // interface faces: free faces between two subdomains, and pressure faces
    std::vector<uint8_t> is_gamma(G.n_faces, 0);
    for (int64_t f = 0; f < G.n_faces; ++f) {
        int ax;
        const int64_t c0 = G.face_cell(f, 0, &ax), c1 = G.face_cell(f, 1, &ax);
        if (I.bct[f] == 1) is_gamma[f] = 1;
        else if (c0 >= 0 && c1 >= 0 && I.part[c0] != I.part[c1]) is_gamma[f] = 1;
    }
    I.gamma.clear();
    for (int64_t f = 0; f < G.n_faces; ++f)
        if (is_gamma[f]) I.gamma.push_back(f);
    for (int s = 0; s < I.N; ++s) {
        Sub& S = I.subs[s];
        std::vector<int64_t> itf, inn;
        for (int64_t c : S.cells)
            for (int a = 0; a < dim; ++a)
                for (int side = 0; side < 2; ++side) {
                    const int64_t f = G.cell_face(c, a, side);
                    if (I.bct[f] == 0) continue;  // no-flow face: not a dof
                    (is_gamma[f] ? itf : inn).push_back(f);
                }
        std::sort(itf.begin(), itf.end());
        itf.erase(std::unique(itf.begin(), itf.end()), itf.end());
        std::sort(inn.begin(), inn.end());
        inn.erase(std::unique(inn.begin(), inn.end()), inn.end());
        S.ng = (int)itf.size();
        S.ni = (int)inn.size();
        S.nc = (int)S.cells.size();
        S.faces = itf;
        S.faces.insert(S.faces.end(), inn.begin(), inn.end());
        S.gidx.resize(S.ng);
        for (int k = 0; k < S.ng; ++k)
            S.gidx[k] = (int)(std::lower_bound(I.gamma.begin(), I.gamma.end(), itf[k]) - I.gamma.begin());
        // per cell-axis local face indices and mass scale
        S.clo.assign((size_t)S.nc * dim, -1);
        S.chi.assign((size_t)S.nc * dim, -1);
        S.cs.assign((size_t)S.nc * dim, 0.0);
        std::vector<int64_t> itf_sorted(itf), inn_sorted(inn);
        auto local = [&](int64_t f) -> int {
            int r = lower_index(itf_sorted, f, 0);
            if (r >= 0) return r;
            r = lower_index(inn_sorted, f, 0);
            return r >= 0 ? S.ng + r : -1;
        };
        for (int r = 0; r < S.nc; ++r) {
            const int64_t c = S.cells[r];
            for (int a = 0; a < dim; ++a) {
                const int64_t fl = G.cell_face(c, a, 0), fu = G.cell_face(c, a, 1);
                S.clo[(size_t)r * dim + a] = (I.bct[fl] == 0) ? -1 : local(fl);
                S.chi[(size_t)r * dim + a] = (I.bct[fu] == 0) ? -1 : local(fu);
                S.cs[(size_t)r * dim + a] = G.h[a] * G.h[a] / G.vol * I.kinv[c * dim + a];
            }
        }
        // face connectivity of the subdomain (through interior faces)
        std::vector<int> parent(S.nc);
        for (int r = 0; r < S.nc; ++r) parent[r] = r;
        std::function<int(int)> find = [&](int x) { while (parent[x] != x) x = parent[x] = parent[parent[x]]; return x; };
        std::vector<int> below(S.ni, -1), above(S.ni, -1);
        for (int r = 0; r < S.nc; ++r)
            for (int a = 0; a < dim; ++a) {
                const int h = S.chi[(size_t)r * dim + a], l = S.clo[(size_t)r * dim + a];
                if (h >= S.ng) below[h - S.ng] = r;
                if (l >= S.ng) above[l - S.ng] = r;
            }
        for (int e = 0; e < S.ni; ++e)
            if (below[e] >= 0 && above[e] >= 0) parent[find(below[e])] = find(above[e]);
        for (int r = 1; r < S.nc; ++r)
            if (find(r) != find(0)) return {BDDC_E_PARTITION, "subdomain " + std::to_string(s) + " is not face-connected"};
    }
    // faces Gamma^{ij} and pressure-face groups
    std::map<std::tuple<int, int, int, int>, int> key2face;
    for (size_t gi = 0; gi < I.gamma.size(); ++gi) {
        const int64_t f = I.gamma[gi];
        int ax;
        const int64_t c0 = G.face_cell(f, 0, &ax), c1 = G.face_cell(f, 1, &ax);
        std::tuple<int, int, int, int> key;
        int owner_lo;  // subdomain that counts +1 (its cell is below the face)
        if (I.bct[f] == 1) {
            const int s = I.part[c0 >= 0 ? c0 : c1];
            key = std::make_tuple(1, s, ax, c1 < 0 ? 1 : 0);
            owner_lo = (c0 >= 0) ? s : -1;
        } else {
            const int p0 = I.part[c0], p1 = I.part[c1];
            key = std::make_tuple(0, std::min(p0, p1), std::max(p0, p1), 0);
            owner_lo = p0;
        }
        auto it = key2face.find(key);
        int fi;
        if (it == key2face.end()) {
            fi = (int)I.faces.size();
            key2face[key] = fi;
            Face F;
            F.dir = std::get<0>(key) == 1;
            F.i = std::get<1>(key);
            F.j = F.dir ? -1 : std::get<2>(key);
            I.faces.push_back(F);
        } else {
            fi = it->second;
        }
        Face& F = I.faces[fi];
        F.gidx.push_back((int)gi);
        F.coef.push_back(owner_lo == F.i ? 1.0 : -1.0);
    }
    // order: shared faces by (i, j), then pressure groups
    std::vector<std::pair<std::tuple<int, int, int, int>, int>> order(key2face.begin(), key2face.end());
    std::vector<Face> sorted;
    for (auto& kv : order) sorted.push_back(I.faces[kv.second]);
    I.faces.swap(sorted);
    int cid = 0;
    for (Face& F : I.faces) {
        F.rows.assign(1, F.coef);
        F.cids.assign(1, cid++);
    }
    I.n_cf = cid;
    return {};
}

// ---- local operators -------------------------------------------------------------
struct Chains {
    std::vector<int> order, start;   // interior indices (0..ni-1) by chain
    std::vector<double> dfac, lfac, off;  // Thomas factors per position; off = coupling to next
};

void build_chains(const Sub& S, int dim, Chains& ch) {
    const int ni = S.ni;
    std::vector<int> below(ni, -1), above(ni, -1), axis(ni, 0);
    for (int r = 0; r < S.nc; ++r)
        for (int a = 0; a < dim; ++a) {
            const int h = S.chi[(size_t)r * dim + a], l = S.clo[(size_t)r * dim + a];
            if (h >= S.ng) { below[h - S.ng] = r; axis[h - S.ng] = a; }
            if (l >= S.ng) { above[l - S.ng] = r; axis[l - S.ng] = a; }
        }
    std::vector<int> next(ni, -1);
    std::vector<uint8_t> has_prev(ni, 0);
    std::vector<double> diag(ni, 0.0), offn(ni, 0.0);
    for (int e = 0; e < ni; ++e) {
        const int a = axis[e];
        const int rb = below[e], ra = above[e];
        diag[e] = kMassDiag * (S.cs[(size_t)rb * dim + a] + S.cs[(size_t)ra * dim + a]);
        const int nx = S.chi[(size_t)ra * dim + a];
        if (nx >= S.ng) {
            next[e] = nx - S.ng;
            offn[e] = kMassOff * S.cs[(size_t)ra * dim + a];
            has_prev[nx - S.ng] = 1;
        }
    }
    ch.order.clear();
    ch.start.clear();
    for (int e = 0; e < ni; ++e) {
        if (has_prev[e]) continue;
        ch.start.push_back((int)ch.order.size());
        for (int x = e; x >= 0; x = next[x]) ch.order.push_back(x);
    }
    ch.start.push_back((int)ch.order.size());
    ch.dfac.resize(ni);
    ch.lfac.resize(ni);
    ch.off.resize(ni);
    for (size_t c = 0; c + 1 < ch.start.size(); ++c) {
        for (int p = ch.start[c]; p < ch.start[c + 1]; ++p) {
            const int e = ch.order[p];
            ch.off[p] = offn[e];
            if (p == ch.start[c]) {
                ch.lfac[p] = 0.0;
                ch.dfac[p] = diag[e];
            } else {
                ch.lfac[p] = ch.off[p - 1] / ch.dfac[p - 1];
                ch.dfac[p] = diag[e] - ch.lfac[p] * ch.off[p - 1];
            }
        }
    }
}

// t = A_II^{-1} x on interior-indexed vectors (in place)
void chain_solve(const Chains& ch, double* x) {
    for (size_t c = 0; c + 1 < ch.start.size(); ++c) {
        const int b = ch.start[c], e = ch.start[c + 1];
        for (int p = b + 1; p < e; ++p) x[ch.order[p]] -= ch.lfac[p] * x[ch.order[p - 1]];
        x[ch.order[e - 1]] /= ch.dfac[e - 1];
        for (int p = e - 2; p >= b; --p)
            x[ch.order[p]] = (x[ch.order[p]] - ch.off[p] * x[ch.order[p + 1]]) / ch.dfac[p];
    }
}

// the cheap part of the local maps: pressure scaling d, sigma, the cell /
// axis / side of every interface dof, and the Thomas factors of A_II
struct LocalPre {
    std::vector<int> gcell, gaxis, gside;
    Chains ch;
};

void local_prologue(const Inst& I, Sub& S, bool pressure_scaling, LocalPre& pre) {
    const int dim = I.geo.dim, ng = S.ng, ni = S.ni, nc = S.nc;
    // diag(A^i) and the pressure scaling d_i (reading: mean of the local
    // unassembled diagonal over all local flux dofs)
    std::vector<double> diagA(ng + ni, 0.0);
    for (int r = 0; r < nc; ++r)
        for (int a = 0; a < dim; ++a) {
            const double s = S.cs[(size_t)r * dim + a];
            const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
            if (l >= 0) diagA[l] += kMassDiag * s;
            if (h >= 0) diagA[h] += kMassDiag * s;
        }
    double sum = 0.0;
    for (double v : diagA) sum += v;
    S.d = (pressure_scaling && ng + ni > 0) ? sum / (ng + ni) : 1.0;
    S.diagA.assign(diagA.begin(), diagA.begin() + ng);
    // sigma = (B^i)^T 1 on interface dofs; the interface dof's cell and side
    std::vector<int> gcell(ng, -1), gaxis(ng, 0), gside(ng, 0);
    for (int r = 0; r < nc; ++r)
        for (int a = 0; a < dim; ++a) {
            const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
            if (l >= 0 && l < ng) { gcell[l] = r; gaxis[l] = a; gside[l] = 0; }
            if (h >= 0 && h < ng) { gcell[h] = r; gaxis[h] = a; gside[h] = 1; }
        }
    S.sigma.resize(ng);
    for (int k = 0; k < ng; ++k) S.sigma[k] = gside[k] == 0 ? 1.0 : -1.0;
    build_chains(S, dim, pre.ch);
    pre.gcell.swap(gcell);
    pre.gaxis.swap(gaxis);
    pre.gside.swap(gside);
}

SetupResult local_maps(const Inst& I, Sub& S, bool pressure_scaling) {
    const int dim = I.geo.dim, ng = S.ng, ni = S.ni, nc = S.nc;
    const double vol = I.geo.vol;
    LocalPre pre;
    local_prologue(I, S, pressure_scaling, pre);
    const double d = S.d;
    const Chains& ch = pre.ch;
    const std::vector<int>&gcell = pre.gcell, &gaxis = pre.gaxis, &gside = pre.gside;
    // Y = A_II^{-1} dB_I^T (ni x nc, column-major per cell)
    std::vector<double> Y((size_t)nc * ni, 0.0);
    for (int r = 0; r < nc; ++r) {
        double* y = &Y[(size_t)r * ni];
        for (int a = 0; a < dim; ++a) {
            const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
            if (l >= ng) y[l - ng] += d;   // B[c, lower] = +1
            if (h >= ng) y[h - ng] -= d;   // B[c, upper] = -1
        }
        chain_solve(ch, y);
    }
    // dB_I t for an interior vector t
    auto dBI = [&](const double* t, double* out) {
        for (int r = 0; r < nc; ++r) {
            double v = 0.0;
            for (int a = 0; a < dim; ++a) {
                const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
                if (l >= ng) v += t[l - ng];
                if (h >= ng) v -= t[h - ng];
            }
            out[r] = d * v;
        }
    };
    // Qm = [[-P, v], [v^T, 0]], P = dB_I Y
    const int nq = nc + 1;
    std::vector<double> Qm((size_t)nq * nq, 0.0);
    std::vector<double> col(nc);
    for (int r = 0; r < nc; ++r) {
        dBI(&Y[(size_t)r * ni], col.data());
        for (int rr = 0; rr < nc; ++rr) Qm[(size_t)rr * nq + r] = -col[rr];
        Qm[(size_t)r * nq + nc] = vol;
        Qm[(size_t)nc * nq + r] = vol;
    }
    std::vector<int> piv;
    if (!lu(nq, Qm.data(), piv)) return {BDDC_E_SETUP, "singular local pressure Schur complement"};

    // solve for the ng + nc input columns, with one step of iterative
    // refinement against the exact sparse local operator (the elimination
    // loses accuracy in proportion to the permeability contrast).  One step
    // suffices: on the 1e7-contrast 60x220 fields a second step changes S^i
    // by 2e-16 and G_post by 6e-12 relative, and the solution's distance to
    // the direct solve of the assembled system not at all.
    const int ncol = ng + nc;
    std::vector<double> XU((size_t)ncol * ni, 0.0);    // interior rhs per column
    std::vector<double> XP((size_t)nq * ncol, 0.0);    // pressure/mu rhs, nq x ncol
    for (int j = 0; j < ng; ++j) {
        const int r = gcell[j], a = gaxis[j];
        const double sc = S.cs[(size_t)r * dim + a];
        // x_u = -A_IG e_j: the other face of the cell along the same axis
        const int other = gside[j] == 0 ? S.chi[(size_t)r * dim + a] : S.clo[(size_t)r * dim + a];
        if (other >= ng) XU[(size_t)j * ni + (other - ng)] = -kMassOff * sc;
        // x_p = -dB_G e_j
        XP[(size_t)r * ncol + j] = -d * (gside[j] == 0 ? 1.0 : -1.0);
    }
    for (int r = 0; r < nc; ++r) XP[(size_t)r * ncol + ng + r] = -d * vol;  // d <f, q_c> per unit f
    // solve K_I [yu; yp; ymu] = [xu; xp; xmu] for all columns
    auto solve_all = [&](const std::vector<double>& xu, const std::vector<double>& xp,
                         std::vector<double>& yu, std::vector<double>& ypm) {
        yu = xu;
        ypm = xp;
        for (int j = 0; j < ncol; ++j) {
            double* t = &yu[(size_t)j * ni];
            chain_solve(ch, t);
            dBI(t, col.data());
            for (int r = 0; r < nc; ++r) ypm[(size_t)r * ncol + j] -= col[r];
        }
        lu_solve(nq, Qm.data(), piv, ypm.data(), ncol);
        // y_u = A_II^{-1} (x_u - dB_I^T y_p): the sparse transpose and a
        // second chain solve (n_i work) in place of the dense product with
        // Y (n_i n_c work)
        for (int j = 0; j < ncol; ++j) {
            double* t = &yu[(size_t)j * ni];
            for (int e = 0; e < ni; ++e) t[e] = xu[(size_t)j * ni + e];
            for (int r = 0; r < nc; ++r) {
                const double yp = ypm[(size_t)r * ncol + j];
                if (yp == 0.0) continue;
                for (int a = 0; a < dim; ++a) {
                    const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
                    if (l >= ng) t[l - ng] -= d * yp;   // B[c, lower] = +1
                    if (h >= ng) t[h - ng] += d * yp;   // B[c, upper] = -1
                }
            }
            chain_solve(ch, t);
        }
    };
    std::vector<double> YU, YPM;
    solve_all(XU, XP, YU, YPM);
    {
        std::vector<double> RU((size_t)ncol * ni), RP((size_t)nq * ncol), DU, DPM;
        for (int pass = 0; pass < kLocalRefinements; ++pass) {
            // residual of K_I y against the right-hand side
            for (int j = 0; j < ncol; ++j) {
                const double* yu = &YU[(size_t)j * ni];
                double* ru = &RU[(size_t)j * ni];
                for (int e = 0; e < ni; ++e) ru[e] = XU[(size_t)j * ni + e];
                double ymu = YPM[(size_t)nc * ncol + j], sump = 0.0;
                for (int r = 0; r < nc; ++r) {
                    const double yp = YPM[(size_t)r * ncol + j];
                    sump += yp;
                    double divr = 0.0;
                    for (int a = 0; a < dim; ++a) {
                        const double sc = S.cs[(size_t)r * dim + a];
                        const int l = S.clo[(size_t)r * dim + a], h = S.chi[(size_t)r * dim + a];
                        const bool li = l >= ng, hi = h >= ng;
                        const double vl = li ? yu[l - ng] : 0.0, vh = hi ? yu[h - ng] : 0.0;
                        if (li) ru[l - ng] -= kMassDiag * sc * vl + kMassOff * sc * vh + d * yp;
                        if (hi) ru[h - ng] -= kMassOff * sc * vl + kMassDiag * sc * vh - d * yp;
                        divr += d * (vl - vh);
                    }
                    RP[(size_t)r * ncol + j] = XP[(size_t)r * ncol + j] - divr - vol * ymu;
                }
                RP[(size_t)nc * ncol + j] = XP[(size_t)nc * ncol + j] - vol * sump;
            }
            solve_all(RU, RP, DU, DPM);
            for (size_t q = 0; q < YU.size(); ++q) YU[q] += DU[q];
            for (size_t q = 0; q < YPM.size(); ++q) YPM[q] += DPM[q];
        }
    }
    // outputs per column
    S.GpostT.assign((size_t)ncol * (ni + nc), 0.0);
    S.S.assign((size_t)ng * ng, 0.0);
    S.GpreT.assign((size_t)nc * ng, 0.0);
    for (int j = 0; j < ncol; ++j) {
        const double* yu = &YU[(size_t)j * ni];
        double* post = &S.GpostT[(size_t)j * (ni + nc)];
        for (int e = 0; e < ni; ++e) post[e] = yu[e];
        for (int r = 0; r < nc; ++r) post[ni + r] = YPM[(size_t)r * ncol + j];
        // interface residual r_G = A_GI y_u + A_GG u_G + dB_G^T y_p
        for (int k = 0; k < ng; ++k) {
            const int r = gcell[k], a = gaxis[k];
            const double sc = S.cs[(size_t)r * dim + a];
            const int other = gside[k] == 0 ? S.chi[(size_t)r * dim + a] : S.clo[(size_t)r * dim + a];
            double v = d * (gside[k] == 0 ? 1.0 : -1.0) * YPM[(size_t)r * ncol + j];
            if (other >= ng) v += kMassOff * sc * yu[other - ng];
            if (j < ng) {
                if (k == j) v += kMassDiag * sc;
                if (other >= 0 && other < ng && other == j) v += kMassOff * sc;
            }
            if (j < ng) S.S[(size_t)j * ng + k] = v;
            else S.GpreT[(size_t)(j - ng) * ng + k] = v;
        }
    }
    for (int a = 0; a < ng; ++a)   // symmetrise S^i (rounding only)
        for (int b = a + 1; b < ng; ++b) {
            const double v = 0.5 * (S.S[(size_t)a * ng + b] + S.S[(size_t)b * ng + a]);
            S.S[(size_t)a * ng + b] = S.S[(size_t)b * ng + a] = v;
        }
    return {};
}

// F_i and Psi_i from S_i and the constraint rows C (m x ng)
SetupResult correction_maps(Sub& S) {
    const int ng = S.ng, m = S.m;
    if (m > ng) return {BDDC_E_SETUP, "more constraints than interface dofs"};
    std::vector<double> Z = null_space(m, ng, S.C.data());
    const int nz = ng - m;
    // ZSZ = Z^T S Z
    std::vector<double> SZ((size_t)ng * nz, 0.0), ZSZ((size_t)nz * nz, 0.0);
    for (int i = 0; i < ng; ++i)
        for (int k = 0; k < ng; ++k) {
            const double s = S.S[(size_t)i * ng + k];
            if (s == 0.0) continue;
            for (int c = 0; c < nz; ++c) SZ[(size_t)i * nz + c] += s * Z[(size_t)k * nz + c];
        }
    for (int a = 0; a < nz; ++a)
        for (int i = 0; i < ng; ++i) {
            const double z = Z[(size_t)i * nz + a];
            for (int b = 0; b < nz; ++b) ZSZ[(size_t)a * nz + b] += z * SZ[(size_t)i * nz + b];
        }
    if (nz > 0 && !chol(nz, ZSZ.data())) return {BDDC_E_SETUP, "constrained local Schur complement not positive definite"};
    // F = Z (ZSZ)^{-1} Z^T
    std::vector<double> W((size_t)nz * ng);   // (ZSZ)^{-1} Z^T
    for (int a = 0; a < nz; ++a)
        for (int i = 0; i < ng; ++i) W[(size_t)a * ng + i] = Z[(size_t)i * nz + a];
    if (nz > 0) chol_solve(nz, ZSZ.data(), W.data(), ng);
    S.F.assign((size_t)ng * ng, 0.0);
    for (int i = 0; i < ng; ++i)
        for (int a = 0; a < nz; ++a) {
            const double z = Z[(size_t)i * nz + a];
            if (z == 0.0) continue;
            for (int j = 0; j < ng; ++j) S.F[(size_t)i * ng + j] += z * W[(size_t)a * ng + j];
        }
    for (int a = 0; a < ng; ++a)
        for (int b = a + 1; b < ng; ++b) {
            const double v = 0.5 * (S.F[(size_t)a * ng + b] + S.F[(size_t)b * ng + a]);
            S.F[(size_t)a * ng + b] = S.F[(size_t)b * ng + a] = v;
        }
    // Psi solves [S C^T; C 0] [Psi; Lam] = [0; I]: Psi = C^+ R2 + Z eta with
    // (Z^T S Z) eta = Z^T (R1 - S C^+ R2), then two steps of iterative
    // refinement against S (the null-space solve loses accuracy in
    // proportion to the conditioning of S)
    std::vector<double> CCt((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            double v = 0.0;
            for (int i = 0; i < ng; ++i) v += S.C[(size_t)a * ng + i] * S.C[(size_t)b * ng + i];
            CCt[(size_t)a * m + b] = v;
        }
    if (m > 0 && !chol(m, CCt.data())) return {BDDC_E_SETUP, "dependent constraint rows"};
    // constrained solve for m right-hand-side columns: R1 (ng x m), R2 (m x m)
    auto csolve = [&](const std::vector<double>& R1, const std::vector<double>& R2, std::vector<double>& X) {
        // y = C^+ R2 = C^T (C C^T)^{-1} R2
        std::vector<double> T(R2);
        if (m > 0) chol_solve(m, CCt.data(), T.data(), m);
        std::vector<double> y((size_t)ng * m, 0.0);
        for (int i = 0; i < ng; ++i)
            for (int a = 0; a < m; ++a) {
                const double c = S.C[(size_t)a * ng + i];
                if (c == 0.0) continue;
                for (int b = 0; b < m; ++b) y[(size_t)i * m + b] += c * T[(size_t)a * m + b];
            }
        // g = R1 - S y ; eta = (Z^T S Z)^{-1} Z^T g
        std::vector<double> g(R1);
        for (int i = 0; i < ng; ++i)
            for (int k = 0; k < ng; ++k) {
                const double sv = S.S[(size_t)i * ng + k];
                if (sv == 0.0) continue;
                for (int b = 0; b < m; ++b) g[(size_t)i * m + b] -= sv * y[(size_t)k * m + b];
            }
        std::vector<double> eta((size_t)nz * m, 0.0);
        for (int c = 0; c < nz; ++c)
            for (int i = 0; i < ng; ++i) {
                const double z = Z[(size_t)i * nz + c];
                if (z == 0.0) continue;
                for (int b = 0; b < m; ++b) eta[(size_t)c * m + b] += z * g[(size_t)i * m + b];
            }
        if (nz > 0) chol_solve(nz, ZSZ.data(), eta.data(), m);
        X = y;
        for (int i = 0; i < ng; ++i)
            for (int c = 0; c < nz; ++c) {
                const double z = Z[(size_t)i * nz + c];
                if (z == 0.0) continue;
                for (int b = 0; b < m; ++b) X[(size_t)i * m + b] += z * eta[(size_t)c * m + b];
            }
    };
    std::vector<double> R1((size_t)ng * m, 0.0), R2((size_t)m * m, 0.0), Psi, dX;
    for (int a = 0; a < m; ++a) R2[(size_t)a * m + a] = 1.0;
    csolve(R1, R2, Psi);
    for (int pass = 0; pass < 2; ++pass) {
        // residuals: R2 = I - C Psi ; R1 = -S Psi projected off the row space of C
        // (the multiplier absorbs the row-space part)
        std::vector<double> SP((size_t)ng * m, 0.0);
        for (int i = 0; i < ng; ++i)
            for (int k = 0; k < ng; ++k) {
                const double sv = S.S[(size_t)i * ng + k];
                if (sv == 0.0) continue;
                for (int b = 0; b < m; ++b) SP[(size_t)i * m + b] += sv * Psi[(size_t)k * m + b];
            }
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) {
                double v = (a == b) ? 1.0 : 0.0;
                for (int i = 0; i < ng; ++i) v -= S.C[(size_t)a * ng + i] * Psi[(size_t)i * m + b];
                R2[(size_t)a * m + b] = v;
            }
        for (size_t q = 0; q < SP.size(); ++q) R1[q] = -SP[q];
        csolve(R1, R2, dX);
        for (size_t q = 0; q < Psi.size(); ++q) Psi[q] += dX[q];
    }
    S.PsiT.assign((size_t)m * ng, 0.0);
    for (int i = 0; i < ng; ++i)
        for (int a = 0; a < m; ++a) S.PsiT[(size_t)a * ng + i] = Psi[(size_t)i * m + a];
    return {};
}

void gather_constraints(Inst& I) {
    for (Sub& S : I.subs) {
        S.C.clear(); S.cid.clear(); S.m = 0; S.rown.clear();
        S.fcs.assign(S.ng, -1);
        S.fcoef.assign(S.ng, 0.0);
    }
    for (const Face& F : I.faces) {
        for (int side = 0; side < (F.dir ? 1 : 2); ++side) {
            Sub& S = I.subs[side == 0 ? F.i : F.j];
            // positions of the face dofs in the subdomain's interface list
            std::vector<int> pos(F.gidx.size());
            for (size_t q = 0; q < F.gidx.size(); ++q)
                pos[q] = (int)(std::lower_bound(S.gidx.begin(), S.gidx.end(), F.gidx[q]) - S.gidx.begin());
            for (size_t rw = 0; rw < F.rows.size(); ++rw) {
                std::vector<double> row(S.ng, 0.0);
                for (size_t q = 0; q < pos.size(); ++q) row[pos[q]] = F.rows[rw][q];
                if (rw == 0)  // the face's net-flux row (Assumption 1)
                    for (size_t q = 0; q < pos.size(); ++q) {
                        S.fcs[pos[q]] = S.m;
                        S.fcoef[pos[q]] = F.rows[0][q];
                    }
                S.rown.push_back(rw == 0 ? (int)pos.size() : 0);
                S.C.insert(S.C.end(), row.begin(), row.end());
                S.cid.push_back(F.cids[rw]);
                S.m++;
            }
        }
    }
}

// Weights of the averaging operator E (Sec. 3), one value per face Gamma^{ij}
// and side: 1/2 (multiplicity), or the face's share of the local diagonals
// sum_F A^i_ee / sum_F (A^i_ee + A^j_ee) (stiffness, Sec. 5); 1 on pressure
// faces.  The Remark "scaling" of Sec. 3: the net-flux constraints keep u*
// conservative only if the weights do not vary along a face; where k jumps
// across the subdomain boundaries only, the per-dof ratios are constant along
// each face and equal these (the rho-scaling of RT0).
void weights(Inst& I, int scaling) {
    // slot of every interface index in each of its (at most two) subdomains
    std::vector<int> sa(I.gamma.size(), -1), sb(I.gamma.size(), -1);
    for (int s = 0; s < (int)I.subs.size(); ++s) {
        Sub& S = I.subs[s];
        S.w.assign(S.ng, 1.0);
        for (int k = 0; k < S.ng; ++k) (sa[S.gidx[k]] < 0 ? sa : sb)[S.gidx[k]] = k;
    }
    for (const Face& F : I.faces) {
        if (F.dir) continue;
        Sub& Si = I.subs[F.i];
        Sub& Sj = I.subs[F.j];
        // the slot of dof g in subdomain X: whichever of sa/sb maps back to g there
        auto slot = [&](const Sub& X, int g) {
            const int a = sa[g];
            return (a >= 0 && a < X.ng && X.gidx[a] == g) ? a : sb[g];
        };
        double wi = 0.5, wj = 0.5;
        if (scaling == BDDC_SCALING_STIFFNESS) {
            double ai = 0.0, aj = 0.0;
            for (int g : F.gidx) {
                ai += Si.diagA[slot(Si, g)];
                aj += Sj.diagA[slot(Sj, g)];
            }
            wi = ai / (ai + aj);
            wj = aj / (ai + aj);
        }
        for (int g : F.gidx) {
            Si.w[slot(Si, g)] = wi;
            Sj.w[slot(Sj, g)] = wj;
        }
    }
}

// modified Gram-Schmidt of `rows` against `basis` (both over the same dofs);
// returns the kept, normalised rows
std::vector<std::vector<double>> orthonormalize(const std::vector<std::vector<double>>& existing,
                                                const std::vector<std::vector<double>>& rows) {
    std::vector<std::vector<double>> basis;
    for (const auto& r : existing) {
        double n = 0.0;
        for (double v : r) n += v * v;
        n = std::sqrt(n);
        std::vector<double> b(r);
        for (double& v : b) v /= n;
        basis.push_back(b);
    }
    std::vector<std::vector<double>> out;
    for (const auto& r : rows) {
        std::vector<double> v(r);
        double n0 = 0.0;
        for (double x : v) n0 += x * x;
        n0 = std::sqrt(n0);
        for (int pass = 0; pass < 2; ++pass)
            for (const auto& b : basis) {
                double dot = 0.0;
                for (size_t q = 0; q < v.size(); ++q) dot += b[q] * v[q];
                for (size_t q = 0; q < v.size(); ++q) v[q] -= dot * b[q];
            }
        double n = 0.0;
        for (double x : v) n += x * x;
        n = std::sqrt(n);
        if (n0 > 0 && n > 1e-10 * n0) {
            for (double& x : v) x /= n;
            basis.push_back(v);
            out.push_back(v);
        }
    }
    return out;
}

// Algorithm 3 on one shared face: returns new rows and omega^{ij}
double adaptive_face(const Inst& I, const Face& F, double tau, std::vector<std::vector<double>>& new_rows) {
    const Sub& Si = I.subs[F.i];
    const Sub& Sj = I.subs[F.j];
    const int f = (int)F.gidx.size();
    std::vector<int> pi(f), pj(f);
    for (int q = 0; q < f; ++q) {
        pi[q] = (int)(std::lower_bound(Si.gidx.begin(), Si.gidx.end(), F.gidx[q]) - Si.gidx.begin());
        pj[q] = (int)(std::lower_bound(Sj.gidx.begin(), Sj.gidx.end(), F.gidx[q]) - Sj.gidx.begin());
    }
    auto Tblock = [&](const Sub& S, const std::vector<int>& p, std::vector<double>& T) {
        std::vector<double> X((size_t)S.ng * f, 0.0);
        for (int q = 0; q < f; ++q) X[(size_t)p[q] * f + q] = 1.0;
        chol_solve(S.ng, S.Lchol.data(), X.data(), f);
        T.assign((size_t)f * f, 0.0);
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) T[(size_t)a * f + b] = X[(size_t)p[a] * f + b];
    };
    std::vector<double> Ti, Tj;
    Tblock(Si, pi, Ti);
    Tblock(Sj, pj, Tj);
    std::vector<double> G((size_t)f * f), SF((size_t)f * f);
    for (int a = 0; a < f; ++a)
        for (int b = 0; b < f; ++b) {
            G[(size_t)a * f + b] = 0.5 * (Ti[(size_t)a * f + b] + Ti[(size_t)b * f + a]) +
                                   0.5 * (Tj[(size_t)a * f + b] + Tj[(size_t)b * f + a]);
            const double wia = Si.w[pi[a]], wib = Si.w[pi[b]], wja = Sj.w[pj[a]], wjb = Sj.w[pj[b]];
            SF[(size_t)a * f + b] = wja * Si.S[(size_t)pi[a] * Si.ng + pi[b]] * wjb +
                                    wia * Sj.S[(size_t)pj[a] * Sj.ng + pj[b]] * wib;
        }
    // face constraints on the jump: c o w_j and c o w_i (one row under
    // multiplicity scaling)
    std::vector<std::vector<double>> crow(2, std::vector<double>(f));
    for (int q = 0; q < f; ++q) {
        crow[0][q] = F.coef[q] * Sj.w[pj[q]];
        crow[1][q] = F.coef[q] * Si.w[pi[q]];
    }
    std::vector<std::vector<double>> cb = orthonormalize({}, crow);
    const int r = (int)cb.size();
    std::vector<double> Cm((size_t)r * f);
    for (int a = 0; a < r; ++a)
        for (int q = 0; q < f; ++q) Cm[(size_t)a * f + q] = cb[a][q];
    std::vector<double> Z = null_space(r, f, Cm.data());
    const int nz = f - r;
    if (nz <= 0) return 0.0;
    // A_r = Z^T S_F Z ; B_r = Z^T G^{-1} Z
    std::vector<double> Lg(G);
    if (!chol(f, Lg.data())) return 0.0;
    std::vector<double> GiZ(Z);
    chol_solve(f, Lg.data(), GiZ.data(), nz);
    std::vector<double> Ar((size_t)nz * nz, 0.0), Br((size_t)nz * nz, 0.0), SFZ((size_t)f * nz, 0.0);
    for (int a = 0; a < f; ++a)
        for (int b = 0; b < f; ++b)
            for (int c = 0; c < nz; ++c) SFZ[(size_t)a * nz + c] += SF[(size_t)a * f + b] * Z[(size_t)b * nz + c];
    for (int x = 0; x < nz; ++x)
        for (int y = 0; y < nz; ++y) {
            double sa = 0.0, sb = 0.0;
            for (int a = 0; a < f; ++a) {
                sa += Z[(size_t)a * nz + x] * SFZ[(size_t)a * nz + y];
                sb += Z[(size_t)a * nz + x] * GiZ[(size_t)a * nz + y];
            }
            Ar[(size_t)x * nz + y] = sa;
            Br[(size_t)x * nz + y] = sb;
        }
    for (int x = 0; x < nz; ++x)
        for (int y = x + 1; y < nz; ++y) {
            Br[(size_t)x * nz + y] = Br[(size_t)y * nz + x] = 0.5 * (Br[(size_t)x * nz + y] + Br[(size_t)y * nz + x]);
            Ar[(size_t)x * nz + y] = Ar[(size_t)y * nz + x] = 0.5 * (Ar[(size_t)x * nz + y] + Ar[(size_t)y * nz + x]);
        }
    if (!chol(nz, Br.data())) return 0.0;
    // M = L^{-1} Ar L^{-T}
    std::vector<double> M(Ar);
    for (int c = 0; c < nz; ++c)        // columns: solve L x = Ar[:, c]
        for (int i = 0; i < nz; ++i) {
            double v = M[(size_t)i * nz + c];
            for (int k = 0; k < i; ++k) v -= Br[(size_t)i * nz + k] * M[(size_t)k * nz + c];
            M[(size_t)i * nz + c] = v / Br[(size_t)i * nz + i];
        }
    for (int rr = 0; rr < nz; ++rr)     // rows: solve L x = M[rr, :]^T
        for (int i = 0; i < nz; ++i) {
            double v = M[(size_t)rr * nz + i];
            for (int k = 0; k < i; ++k) v -= Br[(size_t)i * nz + k] * M[(size_t)rr * nz + k];
            M[(size_t)rr * nz + i] = v / Br[(size_t)i * nz + i];
        }
    for (int x = 0; x < nz; ++x)
        for (int y = x + 1; y < nz; ++y)
            M[(size_t)x * nz + y] = M[(size_t)y * nz + x] = 0.5 * (M[(size_t)x * nz + y] + M[(size_t)y * nz + x]);
    std::vector<double> lam(nz), V((size_t)nz * nz);
    jacobi_eigh(nz, M.data(), lam.data(), V.data());
    std::vector<int> idx(nz);
    for (int q = 0; q < nz; ++q) idx[q] = q;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    int k = 0;
    if (tau > 0 && std::isfinite(tau))
        while (k < nz && lam[idx[k]] > tau) ++k;
    const double omega = k < nz ? std::max(lam[idx[k]], 0.0) : 0.0;
    std::vector<std::vector<double>> rows;
    for (int l = 0; l < k; ++l) {
        // eta = L^{-T} y ; delta = Z eta ; row = S_F delta
        std::vector<double> eta(nz);
        for (int q = 0; q < nz; ++q) eta[q] = V[(size_t)q * nz + idx[l]];
        for (int i = nz - 1; i >= 0; --i) {
            double v = eta[i];
            for (int kk = i + 1; kk < nz; ++kk) v -= Br[(size_t)kk * nz + i] * eta[kk];
            eta[i] = v / Br[(size_t)i * nz + i];
        }
        std::vector<double> delta(f, 0.0), row(f, 0.0);
        for (int a = 0; a < f; ++a)
            for (int q = 0; q < nz; ++q) delta[a] += Z[(size_t)a * nz + q] * eta[q];
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) row[a] += SF[(size_t)a * f + b] * delta[b];
        rows.push_back(row);
    }
    new_rows = orthonormalize(F.rows, rows);
    return omega;
}

// The coarse problem (Sec. 3, eqs. (two-level_coarse-1/2)) in element form:
// per subdomain its coarse dofs (local coarse rows, its pressure, and the
// global-mean multiplier of a pure-flux problem) and the element matrix
// [Psi^T S Psi, d sigma^T Psi; ., 0] (plus d |Omega_i| to the multiplier).
std::vector<CoarseElement> coarse_elements(const Inst& I) {
    const int ncf = I.n_cf, N = I.N;
    const int n = ncf + N + (I.pure ? 1 : 0);
    std::vector<CoarseElement> el(N);
    for (int s = 0; s < N; ++s) {
        const Sub& S = I.subs[s];
        const int ng = S.ng, m = S.m;
        const int e = m + 1 + (I.pure ? 1 : 0);
        CoarseElement& E = el[s];
        E.dofs.assign(S.cid.begin(), S.cid.begin() + m);
        E.dofs.push_back(ncf + s);
        if (I.pure) E.dofs.push_back(n - 1);
        E.E.assign((size_t)e * e, 0.0);
        // Psi^T S Psi and b(psi, 1_s) = d_s sigma^T Psi
        std::vector<double> SP((size_t)m * ng, 0.0);   // (S Psi)^T
        for (int a = 0; a < m; ++a)
            for (int i = 0; i < ng; ++i) {
                double v = 0.0;
                for (int k = 0; k < ng; ++k) v += S.S[(size_t)i * ng + k] * S.PsiT[(size_t)a * ng + k];
                SP[(size_t)a * ng + i] = v;
            }
        for (int a = 0; a < m; ++a) {
            for (int b = 0; b < m; ++b) {
                double v = 0.0;
                for (int i = 0; i < ng; ++i) v += S.PsiT[(size_t)a * ng + i] * SP[(size_t)b * ng + i];
                E.E[(size_t)a * e + b] = v;
            }
            double bv = 0.0;
            for (int i = 0; i < ng; ++i) bv += S.sigma[i] * S.PsiT[(size_t)a * ng + i];
            bv *= S.d;
            E.E[(size_t)m * e + a] = bv;
            E.E[(size_t)a * e + m] = bv;
        }
        if (I.pure) {
            const double v = S.d * S.nc * I.geo.vol;
            E.E[(size_t)m * e + m + 1] = v;
            E.E[(size_t)(m + 1) * e + m] = v;
        }
        // centroid (nested dissection of the sparse coarse factor)
        for (int64_t c : S.cells) {
            const int64_t i = c % I.geo.nx, j = (c / I.geo.nx) % I.geo.ny, k = c / ((int64_t)I.geo.nx * I.geo.ny);
            E.c[0] += (i + 0.5) * I.geo.h[0];
            E.c[1] += (j + 0.5) * I.geo.h[1];
            E.c[2] += (k + 0.5) * I.geo.h[2];
        }
        for (int a = 0; a < 3; ++a) E.c[a] /= (double)std::max<size_t>(1, S.cells.size());
    }
    return el;
}

// dense coarse solver: the inverse of the assembled coarse matrix
SetupResult coarse_dense(Inst& I, const std::vector<CoarseElement>& el) {
    const int ncf = I.n_cf, N = I.N;
    const int n = ncf + N + (I.pure ? 1 : 0);
    std::vector<double> K((size_t)n * n, 0.0);
    for (const CoarseElement& E : el) {
        const int e = (int)E.dofs.size();
        for (int a = 0; a < e; ++a)
            for (int b = 0; b < e; ++b) K[(size_t)E.dofs[a] * n + E.dofs[b]] += E.E[(size_t)a * e + b];
    }
    std::vector<int> piv;
    if (!lu(n, K.data(), piv)) return {BDDC_E_SETUP, "singular coarse problem"};
    std::vector<double> X((size_t)n * n, 0.0);
    lu_inverse(n, K.data(), piv, X.data());
    const int ncn = ncf + N;
    I.Kinv.assign((size_t)ncn * ncn, 0.0);
    for (int a = 0; a < ncn; ++a)
        for (int b = 0; b < ncn; ++b) I.Kinv[(size_t)a * ncn + b] = X[(size_t)a * n + b];
    for (double v : I.Kinv)
        if (!std::isfinite(v)) return {BDDC_E_SETUP, "non-finite coarse inverse"};
    return {};
}

// subdomains per leaf of the coarse dissection tree
constexpr int kCoarseLeafSubdomains = 8;

SetupResult coarse(Inst& I, bool sparse, int nthreads) {
    const std::vector<CoarseElement> el = coarse_elements(I);
    if (!sparse) return coarse_dense(I, el);
    const int n = I.n_cf + I.N + (I.pure ? 1 : 0);
    std::vector<char> is_pressure(n, 0);
    for (int s = 0; s < I.N; ++s) is_pressure[I.n_cf + s] = 1;
    return factor_coarse(n, el, is_pressure, kCoarseLeafSubdomains, nthreads, I.cf);
}

}  // namespace

// make an n x n matrix exactly symmetric: both triangles get the mean of the
// two rounded entries
static void symmetrize(std::vector<double>& M, int n) {
    for (int r = 0; r < n; ++r)
        for (int c = r + 1; c < n; ++c) {
            const double v = 0.5 * (M[(size_t)r * n + c] + M[(size_t)c * n + r]);
            M[(size_t)r * n + c] = v;
            M[(size_t)c * n + r] = v;
        }
}

// the dense part of the local maps of every subdomain on the device: host
// prologues (in parallel), one batch, outputs back into the subdomains
SetupResult device_local_maps(std::vector<Inst>& I, const std::vector<std::pair<int, int>>& tasks, bool ps,
                              int nthreads, LocalMapsDevice device, std::shared_ptr<double>& dev_gpost,
                              int64_t& dev_gpost_count) {
    const int n = (int)tasks.size();
    std::vector<LocalPre> pre(n);
    parallel_for(n, nthreads, [&](int64_t t) {
        auto [b, s] = tasks[t];
        local_prologue(I[b], I[b].subs[s], ps, pre[t]);
    });
    LocalMapsBatch B;
    B.n_sub = n;
    for (auto* v : {&B.o_cell, &B.o_ng, &B.o_ni, &B.o_ch, &B.o_S, &B.o_Gpre, &B.o_Gpost}) v->assign(n + 1, 0);
    for (int t = 0; t < n; ++t) {
        auto [b, s] = tasks[t];
        const Sub& S = I[b].subs[s];
        const int dim = I[b].geo.dim;
        B.dim.push_back(dim);
        B.ng.push_back(S.ng);
        B.ni.push_back(S.ni);
        B.nc.push_back(S.nc);
        B.vol.push_back(I[b].geo.vol);
        B.d.push_back(S.d);
        for (int r = 0; r < S.nc; ++r)
            for (int a = 0; a < 3; ++a) {
                B.clo.push_back(a < dim ? S.clo[(size_t)r * dim + a] : -1);
                B.chi.push_back(a < dim ? S.chi[(size_t)r * dim + a] : -1);
                B.cs.push_back(a < dim ? S.cs[(size_t)r * dim + a] : 0.0);
            }
        B.gcell.insert(B.gcell.end(), pre[t].gcell.begin(), pre[t].gcell.end());
        B.gaxis.insert(B.gaxis.end(), pre[t].gaxis.begin(), pre[t].gaxis.end());
        B.gside.insert(B.gside.end(), pre[t].gside.begin(), pre[t].gside.end());
        const Chains& ch = pre[t].ch;
        B.order.insert(B.order.end(), ch.order.begin(), ch.order.end());
        for (double dv : ch.dfac) B.rdfac.push_back(1.0 / dv);  // the device multiplies
        B.lfac.insert(B.lfac.end(), ch.lfac.begin(), ch.lfac.end());
        B.off.insert(B.off.end(), ch.off.begin(), ch.off.end());
        B.cstart.insert(B.cstart.end(), ch.start.begin(), ch.start.end());
        const int64_t ncol = S.ng + S.nc;
        B.o_cell[t + 1] = B.o_cell[t] + S.nc;
        B.o_ng[t + 1] = B.o_ng[t] + S.ng;
        B.o_ni[t + 1] = B.o_ni[t] + S.ni;
        B.o_ch[t + 1] = B.o_ch[t] + (int64_t)ch.start.size();
        B.o_S[t + 1] = B.o_S[t] + (int64_t)S.ng * S.ng;
        B.o_Gpre[t + 1] = B.o_Gpre[t] + (int64_t)S.nc * S.ng;
        B.o_Gpost[t + 1] = B.o_Gpost[t] + ncol * (S.ni + S.nc);
    }
    std::string err;
    const int rc = device(B, err);
    if (rc) return {rc, "device local maps: " + err};
    for (int t = 0; t < n; ++t) {
        auto [b, s] = tasks[t];
        Sub& S = I[b].subs[s];
        if (B.status[t] != BDDC_OK)
            return {B.status[t], "instance " + std::to_string(b) + " subdomain " + std::to_string(s) +
                                     ": singular local pressure Schur complement"};
        S.S.assign(B.S.begin() + B.o_S[t], B.S.begin() + B.o_S[t + 1]);
        S.GpreT.assign(B.GpreT.begin() + B.o_Gpre[t], B.GpreT.begin() + B.o_Gpre[t + 1]);
        const int ng = S.ng;
        for (int a = 0; a < ng; ++a)  // symmetrise S^i (rounding only)
            for (int c = a + 1; c < ng; ++c) {
                const double v = 0.5 * (S.S[(size_t)a * ng + c] + S.S[(size_t)c * ng + a]);
                S.S[(size_t)a * ng + c] = S.S[(size_t)c * ng + a] = v;
            }
    }
    dev_gpost = B.dev_GpostT;  // G_post stays on the device, in the packed layout
    dev_gpost_count = B.o_Gpost[n];
    return {};
}

// The MsMFEM row of a face Gamma^{ij} (the comparison method of Sec. 5):
// the face flux of the Darcy problem on Omega^i u Omega^j with the sources
// 1/|Omega^i| and -1/|Omega^j| and no flow through the pair's boundary,
// condensed onto the face.  With zero flux on the other interface dofs of
// both subdomains, each subdomain's interface residual is S^k u_F + G_pre^k
// w_k (its local maps); the two pressure constants enter the face rows as
// a multiple of the net-flux row c, and mass balance fixes the net flux
// through the face at int w_i = 1:
//   [S_F  c] [u]   [-g_F]
//   [c^T  0] [l] = [  1 ],   S_F = S^i_FF + S^j_FF, g_F = (G_pre^i w_i - G_pre^j w_j)_F.
// Both subdomains' blocks are in global orientation, so S_F and g_F add.
SetupResult msmfem_face(const Inst& I, const Face& F, std::vector<double>& row) {
    const Sub& Si = I.subs[F.i];
    const Sub& Sj = I.subs[F.j];
    const int f = (int)F.gidx.size();
    std::vector<int> pi(f), pj(f);
    for (int q = 0; q < f; ++q) {
        pi[q] = (int)(std::lower_bound(Si.gidx.begin(), Si.gidx.end(), F.gidx[q]) - Si.gidx.begin());
        pj[q] = (int)(std::lower_bound(Sj.gidx.begin(), Sj.gidx.end(), F.gidx[q]) - Sj.gidx.begin());
    }
    const double wi = 1.0 / ((double)Si.nc * I.geo.vol), wj = 1.0 / ((double)Sj.nc * I.geo.vol);
    const int n = f + 1;
    std::vector<double> K((size_t)n * n, 0.0), rhs(n, 0.0);
    for (int a = 0; a < f; ++a) {
        for (int b = 0; b < f; ++b)
            K[(size_t)a * n + b] = Si.S[(size_t)pi[a] * Si.ng + pi[b]] + Sj.S[(size_t)pj[a] * Sj.ng + pj[b]];
        K[(size_t)a * n + f] = F.coef[a];
        K[(size_t)f * n + a] = F.coef[a];
        double g = 0.0;
        for (int r = 0; r < Si.nc; ++r) g += Si.GpreT[(size_t)r * Si.ng + pi[a]] * wi;
        for (int r = 0; r < Sj.nc; ++r) g -= Sj.GpreT[(size_t)r * Sj.ng + pj[a]] * wj;
        rhs[a] = -g;
    }
    rhs[f] = 1.0;
    std::vector<int> piv;
    if (!lu(n, K.data(), piv)) return {BDDC_E_SETUP, "singular MsMFEM face problem"};
    lu_solve(n, K.data(), piv, rhs.data(), 1);
    row.assign(rhs.begin(), rhs.begin() + f);
    return {};
}

// The caller's constraint rows of an instance, grouped by face: each row
// over the dofs of one face Gamma^{ij} (in the face's dof order).
SetupResult explicit_rows(const Inst& I, std::vector<std::vector<std::vector<double>>>& by_face) {
    by_face.assign(I.faces.size(), {});
    if (I.xrow_ptr.size() < 2) return {};
    // interface index -> (face, position) for the faces between two subdomains
    std::vector<int> gface(I.gamma.size(), -1), gpos(I.gamma.size(), -1);
    for (int fi = 0; fi < (int)I.faces.size(); ++fi) {
        const Face& F = I.faces[fi];
        if (F.dir) continue;
        for (int q = 0; q < (int)F.gidx.size(); ++q) {
            gface[F.gidx[q]] = fi;
            gpos[F.gidx[q]] = q;
        }
    }
    for (size_t r = 0; r + 1 < I.xrow_ptr.size(); ++r) {
        int fi = -1;
        std::vector<double> row;
        for (int64_t q = I.xrow_ptr[r]; q < I.xrow_ptr[r + 1]; ++q) {
            const int64_t face = I.xrow_face[q];
            const auto it = std::lower_bound(I.gamma.begin(), I.gamma.end(), face);
            const int g = (it != I.gamma.end() && *it == face) ? (int)(it - I.gamma.begin()) : -1;
            if (g < 0 || gface[g] < 0 || (fi >= 0 && gface[g] != fi))
                return {BDDC_E_INVALID_ARG, "constraint row " + std::to_string(r) +
                                                " is not on the dofs of one face between two subdomains"};
            if (fi < 0) {
                fi = gface[g];
                row.assign(I.faces[fi].gidx.size(), 0.0);
            }
            row[gpos[g]] += I.xrow_coef[q];
        }
        if (fi >= 0) by_face[fi].push_back(row);
    }
    return {};
}

SetupResult build_all(int n_inst, const bddc_instance* inst, const bddc_options& opt, Packed& P,
                      LocalMapsDevice device, FaceEigenDevice eig_device) {
    const int nthreads = opt.n_threads > 0 ? opt.n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    TraceStage stage("bddc_setup: instances and topology");
    std::vector<Inst> I(n_inst);
    {
        std::vector<SetupResult> rr(n_inst);
        parallel_for(n_inst, nthreads, [&](int64_t b) {
            rr[b] = read_instance(inst[b], I[b]);
            if (!rr[b].code) rr[b] = build_topology(I[b]);
        });
        for (int b = 0; b < n_inst; ++b)
            if (rr[b].code) { rr[b].msg = "instance " + std::to_string(b) + ": " + rr[b].msg; return rr[b]; }
    }
    // flat task list over all subdomains
    std::vector<std::pair<int, int>> tasks;
    for (int b = 0; b < n_inst; ++b)
        for (int s = 0; s < I[b].N; ++s) tasks.emplace_back(b, s);
    std::mutex mu;
    SetupResult err;
    auto fail = [&](const SetupResult& r, int b, int s) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err.code) err = {r.code, "instance " + std::to_string(b) + " subdomain " + std::to_string(s) + ": " + r.msg};
    };
    std::shared_ptr<double> dev_gpost;
    int64_t dev_gpost_count = 0;
    stage.next("bddc_setup: local maps");
    if (device) {
        SetupResult r = device_local_maps(I, tasks, opt.pressure_scaling != 0, nthreads, device, dev_gpost,
                                          dev_gpost_count);
        if (r.code) return r;
    } else {
        parallel_for((int64_t)tasks.size(), nthreads, [&](int64_t t) {
            auto [b, s] = tasks[t];
            SetupResult r = local_maps(I[b], I[b].subs[s], opt.pressure_scaling != 0);
            if (r.code) fail(r, b, s);
        });
        if (err.code) return err;
    }
    stage.next("bddc_setup: weights and constraints (Algorithm 3)");
    for (int b = 0; b < n_inst; ++b) weights(I[b], opt.scaling);
    const bool adaptive = opt.constraints == BDDC_CONSTRAINTS_ADAPTIVE && opt.tau > 0 && std::isfinite(opt.tau);
    const bool add_rows = adaptive || opt.constraints != BDDC_CONSTRAINTS_ADAPTIVE;
    {
        std::vector<std::pair<int, int>> ftasks;
        for (int b = 0; b < n_inst; ++b)
            for (int fi = 0; fi < (int)I[b].faces.size(); ++fi)
                if (!I[b].faces[fi].dir) ftasks.emplace_back(b, fi);
        std::vector<std::vector<std::vector<double>>> rows(ftasks.size());
        std::vector<double> om(ftasks.size(), 0.0);
        if (eig_device && !ftasks.empty()) {
            // the face eigenproblems on the GPU, batched over all faces (the
            // rows are orthonormalised against the face's rows here)
            FaceEigenBatch B;
            std::vector<int64_t> sub0(n_inst + 1, 0);
            for (int b = 0; b < n_inst; ++b) sub0[b + 1] = sub0[b] + I[b].N;
            B.n.resize(sub0[n_inst]);
            B.o_S.assign(1, 0);
            B.o_w.assign(1, 0);
            for (int b = 0; b < n_inst; ++b)
                for (int q = 0; q < I[b].N; ++q) {
                    const Sub& S = I[b].subs[q];
                    B.n[sub0[b] + q] = S.ng;
                    B.o_S.push_back(B.o_S.back() + (int64_t)S.ng * S.ng);
                    B.o_w.push_back(B.o_w.back() + S.ng);
                }
            B.S.resize(B.o_S.back());
            B.w.resize(B.o_w.back());
            parallel_for(n_inst, nthreads, [&](int64_t b) {
                for (int q = 0; q < I[b].N; ++q) {
                    const Sub& S = I[b].subs[q];
                    std::copy(S.S.begin(), S.S.end(), B.S.begin() + B.o_S[sub0[b] + q]);
                    std::copy(S.w.begin(), S.w.end(), B.w.begin() + B.o_w[sub0[b] + q]);
                }
            });
            B.o_f.assign(1, 0);
            B.o_rows.assign(1, 0);
            for (auto [b, fi] : ftasks) {
                const Face& F = I[b].faces[fi];
                const Sub& Si = I[b].subs[F.i];
                const Sub& Sj = I[b].subs[F.j];
                const int f = (int)F.gidx.size();
                B.fi.push_back((int)(sub0[b] + F.i));
                B.fj.push_back((int)(sub0[b] + F.j));
                B.ff.push_back(f);
                for (int q = 0; q < f; ++q) {
                    B.pi.push_back((int)(std::lower_bound(Si.gidx.begin(), Si.gidx.end(), F.gidx[q]) - Si.gidx.begin()));
                    B.pj.push_back((int)(std::lower_bound(Sj.gidx.begin(), Sj.gidx.end(), F.gidx[q]) - Sj.gidx.begin()));
                    B.coef.push_back(F.coef[q]);
                }
                B.o_f.push_back(B.o_f.back() + f);
                B.o_rows.push_back(B.o_rows.back() + (int64_t)f * f);
            }
            B.tau = adaptive ? opt.tau : -1.0;
            std::string msg;
            const int rc = eig_device(B, msg);
            if (rc) return {rc, "face eigenproblems on the device: " + msg};
            parallel_for((int64_t)ftasks.size(), nthreads, [&](int64_t t) {
                auto [b, fi] = ftasks[t];
                const Face& F = I[b].faces[fi];
                const int f = B.ff[t];
                std::vector<std::vector<double>> raw(B.nrows[t], std::vector<double>(f));
                for (int l = 0; l < B.nrows[t]; ++l)
                    std::copy(B.rows.begin() + B.o_rows[t] + (int64_t)l * f,
                              B.rows.begin() + B.o_rows[t] + (int64_t)(l + 1) * f, raw[l].begin());
                om[t] = B.omega[t];
                rows[t] = orthonormalize(F.rows, raw);
            });
        } else {
            // Cholesky of every S^i (the face problems need (S^i)^{-1}); always
            // done so that omega-tilde is reported for the initial constraints too
            parallel_for((int64_t)tasks.size(), nthreads, [&](int64_t t) {
                auto [b, s] = tasks[t];
                Sub& S = I[b].subs[s];
                S.Lchol = S.S;
                if (!chol(S.ng, S.Lchol.data())) fail({BDDC_E_SETUP, "interface Schur complement not positive definite"}, b, s);
            });
            if (err.code) return err;
            parallel_for((int64_t)ftasks.size(), nthreads, [&](int64_t t) {
                auto [b, fi] = ftasks[t];
                om[t] = adaptive_face(I[b], I[b].faces[fi], adaptive ? opt.tau : -1.0, rows[t]);
            });
        }
        // the other constraint modes: MsMFEM rows or the caller's rows
        // (Algorithm 3 above still gives omega-tilde of the initial constraints)
        if (opt.constraints == BDDC_CONSTRAINTS_MSMFEM) {
            std::vector<SetupResult> fres(ftasks.size());
            parallel_for((int64_t)ftasks.size(), nthreads, [&](int64_t t) {
                auto [b, fi] = ftasks[t];
                std::vector<double> row;
                fres[t] = msmfem_face(I[b], I[b].faces[fi], row);
                rows[t] = fres[t].code ? std::vector<std::vector<double>>{}
                                       : orthonormalize(I[b].faces[fi].rows, {row});
            });
            for (auto& r : fres)
                if (r.code) return r;
        } else if (opt.constraints == BDDC_CONSTRAINTS_EXPLICIT) {
            std::vector<std::vector<std::vector<std::vector<double>>>> xr(n_inst);
            for (int b = 0; b < n_inst; ++b) {
                SetupResult r = explicit_rows(I[b], xr[b]);
                if (r.code) {
                    r.msg = "instance " + std::to_string(b) + ": " + r.msg;
                    return r;
                }
            }
            parallel_for((int64_t)ftasks.size(), nthreads, [&](int64_t t) {
                auto [b, fi] = ftasks[t];
                rows[t] = xr[b][fi].empty() ? std::vector<std::vector<double>>{}
                                            : orthonormalize(I[b].faces[fi].rows, xr[b][fi]);
            });
        }
        for (size_t t = 0; t < ftasks.size(); ++t) {
            auto [b, fi] = ftasks[t];
            I[b].omega = std::max(I[b].omega, om[t]);
            if (!add_rows) continue;
            Face& F = I[b].faces[fi];
            for (auto& r : rows[t]) {
                F.rows.push_back(r);
                F.cids.push_back(I[b].n_cf++);
                I[b].n_adapt++;
            }
        }
    }
    for (int b = 0; b < n_inst; ++b) gather_constraints(I[b]);
    stage.next("bddc_setup: correction maps");
    parallel_for((int64_t)tasks.size(), nthreads, [&](int64_t t) {
        auto [b, s] = tasks[t];
        SetupResult r = correction_maps(I[b].subs[s]);
        if (r.code) fail(r, b, s);
    });
    if (err.code) return err;
    // coarse solver: dense inverse, or the sparse factor for large coarse problems
    stage.next("bddc_setup: coarse solver");
    int max_ncn = 0;
    for (int b = 0; b < n_inst; ++b) max_ncn = std::max(max_ncn, I[b].n_cf + I[b].N);
    const bool sparse = opt.coarse_solver == BDDC_COARSE_SPARSE ||
                        (opt.coarse_solver == BDDC_COARSE_AUTO && max_ncn > BDDC_COARSE_DENSE_MAX);
    std::vector<SetupResult> cres(n_inst);
    if (sparse) {
        for (int b = 0; b < n_inst; ++b) cres[b] = coarse(I[b], true, nthreads);
    } else {
        parallel_for(n_inst, nthreads, [&](int64_t b) { cres[b] = coarse(I[b], false, 1); });
    }
    for (int b = 0; b < n_inst; ++b)
        if (cres[b].code) { cres[b].msg = "instance " + std::to_string(b) + ": " + cres[b].msg; return cres[b]; }

    // ---- pack -----------------------------------------------------------------
    stage.next("bddc_setup: pack");
    P = Packed();
    P.precision = opt.precision;
    P.dev_Gpost = dev_gpost;  // set: G_post is on the device and P.Gpost stays empty
    P.dev_Gpost_count = dev_gpost_count;
    int64_t goff = 0, coff = 0, kinv_off = 0, s_glob = 0, face_off = 0, cell_off = 0;
    int64_t slot = 0, cslot = 0, celll = 0, intl = 0;
    int64_t oS = 0, oF = 0, oP = 0, oGpre = 0, oGpost = 0;
    P.off_slot.push_back(0); P.off_cslot.push_back(0); P.off_cell.push_back(0); P.off_int.push_back(0);
    for (int b = 0; b < n_inst; ++b) {
        Inst& In = I[b];
        const int ncn = In.n_cf + In.N;
        P.inst_goff.push_back(goff); P.inst_ng.push_back((int64_t)In.gamma.size());
        P.inst_coff.push_back(coff); P.inst_ncn.push_back(ncn); P.inst_ncf.push_back(In.n_cf);
        P.inst_kinv_off.push_back(kinv_off);
        P.inst_s0.push_back(s_glob); P.inst_s1.push_back(s_glob + In.N);
        P.inst_face_off.push_back(face_off); P.inst_nfaces.push_back(In.geo.n_faces);
        P.inst_cell_off.push_back(cell_off); P.inst_ncells.push_back(In.geo.n_cells);
        P.inst_vol.push_back(In.geo.vol);
        P.inst_nadapt.push_back(In.n_adapt);
        P.inst_omega.push_back(In.omega);
        P.inst_grid.insert(P.inst_grid.end(), {In.geo.dim, In.geo.nx, In.geo.ny, In.geo.nz});
        P.inst_h.insert(P.inst_h.end(), {In.geo.h[0], In.geo.h[1], In.geo.h[2]});
        for (int64_t c = 0; c < In.geo.n_cells; ++c)
            for (int a = 0; a < 3; ++a) P.cell_kinv.push_back(a < In.geo.dim ? In.kinv[(size_t)c * In.geo.dim + a] : 0.0);
        P.face_bct.insert(P.face_bct.end(), In.bct.begin(), In.bct.end());
        P.max_ncn = std::max(P.max_ncn, ncn);
        // per interface dof
        const int64_t ngam = (int64_t)In.gamma.size();
        std::vector<int> sa(ngam, -1), sb(ngam, -1);
        for (int64_t q = 0; q < ngam; ++q) {
            const int64_t f = In.gamma[q];
            P.g_fid.push_back(face_off + f);
            int ax;
            double sign = 0.0;
            if (In.bct[f] == 1) sign = In.geo.face_cell(f, 1, &ax) < 0 ? -1.0 : 1.0;
            P.g_bsign.push_back(sign);
        }
        std::vector<int> ca((size_t)In.n_cf, -1), cb((size_t)In.n_cf, -1);
        for (int s = 0; s < In.N; ++s) {
            Sub& S = In.subs[s];
            P.sub_inst.push_back(b); P.sub_ng.push_back(S.ng); P.sub_ni.push_back(S.ni);
            P.sub_nc.push_back(S.nc); P.sub_m.push_back(S.m); P.sub_local.push_back(s);
            P.sub_d.push_back(S.d);
            P.max_ng = std::max(P.max_ng, S.ng);
            P.max_m = std::max(P.max_m, S.m);
            P.max_out_post = std::max(P.max_out_post, S.ni + S.nc);
            P.max_in_post = std::max(P.max_in_post, S.ng + S.nc);
            P.off_S.push_back(oS); P.off_F.push_back(oF); P.off_P.push_back(oP);
            P.off_Gpre.push_back(oGpre); P.off_Gpost.push_back(oGpost);
            // every operator block starts on a multiple of 4 elements (16-byte
            // alignment for FP32, 32 for FP64) and is zero-padded to one, so
            // a block can be copied whole by a 1D bulk copy
            auto pad4 = [](int64_t n) { return (n + 3) & ~(int64_t)3; };
            const int64_t nS = (int64_t)S.ng * S.ng, nP = (int64_t)S.m * S.ng;
            // the operator blocks are copied after this loop, in parallel, at
            // these offsets
            oS += pad4(nS);
            oF += pad4(nS);
            oP += pad4(nP);
            oGpre += (int64_t)S.nc * S.ng;
            oGpost += (int64_t)(S.ng + S.nc) * (S.ni + S.nc);
            for (int k = 0; k < S.ng; ++k) {
                const int g = S.gidx[k];
                P.slot_g.push_back((int)(goff + g));
                P.slot_w.push_back(S.w[k]);
                P.slot_dsig.push_back(S.d * S.sigma[k]);
                P.slot_fcs.push_back(S.fcs[k]);
                P.slot_coef.push_back(S.fcoef[k]);
                if (sa[g] < 0) sa[g] = (int)(slot + k); else sb[g] = (int)(slot + k);
            }
            if (opt.formulation == BDDC_FORM_FULL) {
                // full-space form: the cell of S on each interface face and
                // that cell's other face along the face's axis (S.faces holds
                // the interface faces sorted, then the interior ones sorted;
                // S.cells is sorted)
                auto face_pos = [&](int64_t f) -> int {
                    auto it = std::lower_bound(S.faces.begin(), S.faces.begin() + S.ng, f);
                    if (it != S.faces.begin() + S.ng && *it == f) return (int)(it - S.faces.begin());
                    it = std::lower_bound(S.faces.begin() + S.ng, S.faces.end(), f);
                    if (it != S.faces.end() && *it == f) return (int)(it - S.faces.begin());
                    return -1;
                };
                auto cell_pos = [&](int64_t c) -> int {
                    if (c < 0) return -1;
                    const auto it = std::lower_bound(S.cells.begin(), S.cells.end(), c);
                    return (it != S.cells.end() && *it == c) ? (int)(it - S.cells.begin()) : -1;
                };
                for (int k = 0; k < S.ng; ++k) {
                    const int64_t f = S.faces[k];
                    int ax = 0;
                    int64_t K = In.geo.face_cell(f, 1, &ax);  // the cell above f
                    int r = cell_pos(K);
                    const bool lower = r >= 0;
                    if (!lower) {
                        K = In.geo.face_cell(f, 0, &ax);
                        r = cell_pos(K);
                    }
                    if (r < 0) return {BDDC_E_SETUP, "interface face without a cell of its subdomain"};
                    const int64_t opp = In.geo.cell_face(K, ax, lower ? 1 : 0);
                    const int o = face_pos(opp);
                    if (o < 0 && In.bct[opp] != 0)
                        return {BDDC_E_SETUP, "a cell face that is neither a subdomain unknown nor a no-flow face"};
                    P.slot_fopp.push_back(o);
                    P.slot_fcell.push_back(lower ? r + 1 : -(r + 1));
                    P.slot_fk.push_back(In.geo.h[ax] * In.geo.h[ax] / In.geo.vol * In.kinv[(size_t)K * In.geo.dim + ax]);
                }
            }
            {
                int start = 0;
                for (int a = 0; a < S.m; ++a) {
                    if (S.rown[a] == 0) { P.cslot_fstart.push_back(-1); continue; }
                    P.cslot_fstart.push_back(start);
                    for (int k = 0; k < S.ng; ++k)
                        if (S.fcs[k] == a) {
                            P.slot_fperm.push_back(k);
                            P.slot_fcoefp.push_back(S.fcoef[k]);
                            ++start;
                        }
                }
            }
            for (int a = 0; a < S.m; ++a) {
                P.cslot_c.push_back(S.cid[a]);
                P.cslot_n.push_back(S.rown[a]);
                const int c = S.cid[a];
                if (ca[c] < 0) ca[c] = (int)(cslot + a); else cb[c] = (int)(cslot + a);
            }
            for (int r = 0; r < S.nc; ++r) P.cell_gid.push_back(cell_off + S.cells[r]);
            for (int e = 0; e < S.ni; ++e) P.int_fid.push_back(face_off + S.faces[S.ng + e]);
            slot += S.ng; cslot += S.m; celll += S.nc; intl += S.ni;
            P.off_slot.push_back(slot); P.off_cslot.push_back(cslot);
            P.off_cell.push_back(celll); P.off_int.push_back(intl);
        }
        for (int64_t q = 0; q < ngam; ++q) { P.g_slot_a.push_back(sa[q]); P.g_slot_b.push_back(sb[q]); }
        for (int c = 0; c < In.n_cf; ++c) { P.c_slot_a.push_back(ca[c]); P.c_slot_b.push_back(cb[c]); }
        goff += ngam; coff += ncn; kinv_off += (int64_t)In.Kinv.size(); s_glob += In.N;
        face_off += In.geo.n_faces; cell_off += In.geo.n_cells;
    }
    // the operator blocks and coarse inverses, copied in parallel into arrays
    // sized once (zero padding included).  S and F are symmetric in exact
    // arithmetic; they are stored exactly symmetric (mean of the two rounded
    // triangles) so that one triangle describes each.
    {
        std::vector<std::pair<int, int>> subs;
        for (int b = 0; b < n_inst; ++b)
            for (int q = 0; q < I[b].N; ++q) subs.emplace_back(b, q);
        const bool fp32 = opt.precision == BDDC_PREC_FP32;
        P.S.assign((size_t)oS, 0.0);
        P.P64.assign((size_t)oP, 0.0);
        if (fp32) {
            P.F32.assign((size_t)oF, 0.0f);
            P.P32.assign((size_t)oP, 0.0f);
        } else {
            P.F64.assign((size_t)oF, 0.0);
        }
        P.Gpre.assign((size_t)oGpre, 0.0);
        if (!P.dev_Gpost) P.Gpost.assign((size_t)oGpost, 0.0);
        parallel_for((int64_t)subs.size(), nthreads, [&](int64_t g) {
            Sub& S = I[subs[g].first].subs[subs[g].second];
            symmetrize(S.S, S.ng);
            symmetrize(S.F, S.ng);
            std::copy(S.S.begin(), S.S.end(), P.S.begin() + P.off_S[g]);
            std::copy(S.PsiT.begin(), S.PsiT.end(), P.P64.begin() + P.off_P[g]);
            if (fp32) {
                std::transform(S.F.begin(), S.F.end(), P.F32.begin() + P.off_F[g], [](double v) { return (float)v; });
                std::transform(S.PsiT.begin(), S.PsiT.end(), P.P32.begin() + P.off_P[g], [](double v) { return (float)v; });
            } else {
                std::copy(S.F.begin(), S.F.end(), P.F64.begin() + P.off_F[g]);
            }
            std::copy(S.GpreT.begin(), S.GpreT.end(), P.Gpre.begin() + P.off_Gpre[g]);
            if (!P.dev_Gpost) std::copy(S.GpostT.begin(), S.GpostT.end(), P.Gpost.begin() + P.off_Gpost[g]);
        });
        P.Kinv.assign((size_t)kinv_off, 0.0);
        parallel_for(n_inst, nthreads, [&](int64_t b) {
            std::copy(I[b].Kinv.begin(), I[b].Kinv.end(), P.Kinv.begin() + P.inst_kinv_off[b]);
        });
    }
    // slot partner (the other copy of the same interface dof)
    P.slot_partner.assign(slot, -1);
    for (size_t q = 0; q < P.g_slot_a.size(); ++q)
        if (P.g_slot_b[q] >= 0) {
            P.slot_partner[P.g_slot_a[q]] = P.g_slot_b[q];
            P.slot_partner[P.g_slot_b[q]] = P.g_slot_a[q];
        }
    P.n_sub = s_glob;
    P.n_gamma = goff;
    P.n_coarse_vec = coff;
    if (sparse) {
        // the multifrontal factors of all instances, batched
        P.coarse_sparse = 1;
        int64_t csoff = 0, u_off = 0, dof_off = 0, xo = 0, ho = 0;
        for (int b = 0; b < n_inst; ++b) {
            const CoarseFactor& cf = I[b].cf;
            const int nn = (int)cf.piv.size();
            P.inst_csoff.push_back(csoff);
            P.inst_node0.push_back((int64_t)P.cn_p.size());
            std::vector<int64_t> uo(nn);
            for (int v = 0; v < nn; ++v) {
                uo[v] = u_off;
                u_off += (int64_t)cf.bnd[v].size();
            }
            auto child_pos = [&](int c, int d) -> int {
                if (c < 0) return -1;
                const std::vector<int>& cb = cf.bnd[c];
                const auto it = std::lower_bound(cb.begin(), cb.end(), d);
                return (it != cb.end() && *it == d) ? (int)(uo[c] + (it - cb.begin())) : -1;
            };
            for (int v = 0; v < nn; ++v) {
                const int p = (int)cf.piv[v].size(), q = (int)cf.bnd[v].size();
                P.cn_inst.push_back(b);
                P.cn_p.push_back(p);
                P.cn_q.push_back(q);
                P.cn_depth.push_back(cf.depth[v]);
                P.cn_off_dof.push_back(dof_off);
                P.cn_off_X.push_back(xo);
                P.cn_off_H.push_back(ho);
                P.cn_off_u.push_back(uo[v]);
                for (int pass = 0; pass < 2; ++pass)
                    for (int d : pass ? cf.bnd[v] : cf.piv[v]) {
                        P.cn_dof.push_back(d);
                        P.cn_c0.push_back(child_pos(cf.child0[v], d));
                        P.cn_c1.push_back(child_pos(cf.child1[v], d));
                    }
                P.cn_X.insert(P.cn_X.end(), cf.X[v].begin(), cf.X[v].end());
                P.cn_H.insert(P.cn_H.end(), cf.H[v].begin(), cf.H[v].end());
                for (int j = 0; j < q; ++j)
                    for (int i = 0; i < p; ++i) P.cn_HT.push_back(cf.H[v][(size_t)i * q + j]);
                dof_off += p + q;
                xo += (int64_t)p * p;
                ho += (int64_t)p * q;
            }
            P.cn_max_depth = std::max(P.cn_max_depth, cf.max_depth);
            csoff += cf.n;
        }
        P.inst_csoff.push_back(csoff);
        P.inst_node0.push_back((int64_t)P.cn_p.size());
        P.n_csys = csoff;
        P.n_cu = u_off;
    }
    return {};
}

}  // namespace bddc

// ---- host-only inspection ------------------------------------------------------
struct bddc_host_setup {
    bddc::Packed P;
};

// message of the last failed setup of this thread (bddc_last_error(NULL))
extern thread_local std::string g_setup_err;

namespace {
template <class T>
bool export_vec(const std::vector<T>& v, void* dst, int64_t* count, int* eb) {
    if (count) *count = (int64_t)v.size();
    if (eb) *eb = (int)sizeof(T);
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(T));
    return true;
}

bool export_named(const bddc::Packed& P, const char* name, void* dst, int64_t* count, int* eb) {
    const std::string n(name ? name : "");
    if (n == "Gpost" && P.dev_Gpost) {
        if (count) *count = P.dev_Gpost_count;
        if (eb) *eb = 8;
        return !dst || bddc::device_to_host(P.dev_Gpost.get(), P.dev_Gpost_count, static_cast<double*>(dst));
    }
#define E(x) if (n == #x) return export_vec(P.x, dst, count, eb)
    E(sub_inst); E(sub_ng); E(sub_ni); E(sub_nc); E(sub_m); E(sub_local); E(slot_g); E(slot_partner);
    E(cslot_c); E(c_slot_a); E(c_slot_b); E(g_slot_a); E(g_slot_b); E(slot_fcs); E(cslot_n); E(slot_coef); E(slot_fperm); E(cslot_fstart); E(slot_fcoefp);
    E(inst_goff); E(inst_ng); E(inst_coff); E(inst_ncn); E(inst_ncf); E(inst_kinv_off); E(inst_s0); E(inst_s1);
    E(inst_face_off); E(inst_nfaces); E(inst_cell_off); E(inst_ncells); E(off_S); E(off_F); E(off_P);
    E(off_Gpre); E(off_Gpost); E(off_slot); E(off_cslot); E(off_cell); E(off_int); E(cell_gid); E(int_fid); E(g_fid);
    E(inst_vol); E(inst_omega); E(sub_d); E(slot_w); E(slot_dsig); E(g_bsign); E(S); E(Gpre); E(Gpost); E(Kinv); E(P64);
    E(slot_fk); E(slot_fopp); E(slot_fcell);
    E(inst_csoff); E(inst_node0); E(cn_inst); E(cn_p); E(cn_q); E(cn_depth); E(cn_off_dof); E(cn_off_X); E(cn_off_H);
    E(cn_off_u); E(cn_dof); E(cn_c0); E(cn_c1); E(cn_X); E(cn_H); E(cn_HT);
#undef E
    if (n == "F" || n == "P") {
        const bool isF = n == "F";
        const std::vector<double>& v64 = isF ? P.F64 : (P.P32.empty() ? P.P64 : std::vector<double>());
        const std::vector<float>& v32 = isF ? P.F32 : P.P32;
        if (!v64.empty()) return export_vec(v64, dst, count, eb);
        if (count) *count = (int64_t)v32.size();
        if (eb) *eb = 8;
        if (dst) {
            double* d = static_cast<double*>(dst);
            for (size_t q = 0; q < v32.size(); ++q) d[q] = v32[q];
        }
        return true;
    }
    if (count) *count = 0;
    if (eb) *eb = 0;
    return false;
}
// x = K_c^{-1} rhs for instance b with the packed coarse solver (dense
// inverse, or the multifrontal sweeps over the packed factor exactly as the
// device runs them); rhs and x have n_c + N entries
void packed_coarse_solve(const bddc::Packed& P, int b, const double* rhs, double* x) {
    const int64_t ncn = P.inst_ncn[b];
    if (!P.coarse_sparse) {
        const double* K = P.Kinv.data() + P.inst_kinv_off[b];
        for (int64_t r = 0; r < ncn; ++r) {
            double acc = 0.0;
            for (int64_t c = 0; c < ncn; ++c) acc += K[r * ncn + c] * rhs[c];
            x[r] = acc;
        }
        return;
    }
    const int64_t n = P.inst_csoff[b + 1] - P.inst_csoff[b];
    std::vector<double> bb(n, 0.0), t(n, 0.0), xx(n, 0.0), u(P.n_cu, 0.0);
    for (int64_t c = 0; c < ncn; ++c) bb[c] = rhs[c];
    const int64_t v0 = P.inst_node0[b], v1 = P.inst_node0[b + 1];
    auto upd = [&](int c) { return c >= 0 ? u[c] : 0.0; };
    for (int64_t v = v0; v < v1; ++v) {
        const int p = P.cn_p[v], q = P.cn_q[v];
        const int64_t od = P.cn_off_dof[v], oh = P.cn_off_H[v], ou = P.cn_off_u[v];
        for (int i = 0; i < p; ++i) {
            const int d = P.cn_dof[od + i];
            t[d] = bb[d] + upd(P.cn_c0[od + i]) + upd(P.cn_c1[od + i]);
        }
        for (int j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int i = 0; i < p; ++i) acc += P.cn_H[oh + (int64_t)i * q + j] * t[P.cn_dof[od + i]];
            u[ou + j] = upd(P.cn_c0[od + p + j]) + upd(P.cn_c1[od + p + j]) - acc;
        }
    }
    for (int64_t v = v1 - 1; v >= v0; --v) {
        const int p = P.cn_p[v], q = P.cn_q[v];
        const int64_t od = P.cn_off_dof[v], ox = P.cn_off_X[v], oh = P.cn_off_H[v];
        for (int i = 0; i < p; ++i) {
            double acc = 0.0;
            for (int k = 0; k < p; ++k) acc += P.cn_X[ox + (int64_t)k * p + i] * t[P.cn_dof[od + k]];
            for (int j = 0; j < q; ++j) acc -= P.cn_HT[oh + (int64_t)j * p + i] * xx[P.cn_dof[od + p + j]];
            xx[P.cn_dof[od + i]] = acc;
        }
    }
    for (int64_t c = 0; c < ncn; ++c) x[c] = xx[c];
}
}  // namespace

extern "C" {

int bddc_host_setup_coarse_solve(const bddc_host_setup* hs, int instance, const double* rhs, double* x) {
    if (!hs || !rhs || !x || instance < 0 || instance >= (int)hs->P.inst_ncn.size()) return BDDC_E_INVALID_ARG;
    packed_coarse_solve(hs->P, instance, rhs, x);
    return BDDC_OK;
}

static int host_setup_create(int n_instances, const bddc_instance* inst, const bddc_options* opt_in,
                             bddc_host_setup** out, bddc::LocalMapsDevice device) {
    if (!out) return BDDC_E_INVALID_ARG;
    *out = nullptr;
    if (n_instances <= 0 || !inst) return BDDC_E_INVALID_ARG;
    bddc_options opt;
    bddc_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (!bddc::options_valid(opt)) return BDDC_E_INVALID_ARG;
    auto* hs = new bddc_host_setup();
    bddc::SetupResult r = bddc::build_all(n_instances, inst, opt, hs->P, device, device ? bddc::face_eigen_device : nullptr);
    if (r.code) {
        g_setup_err = r.msg;
        delete hs;
        return r.code;
    }
    *out = hs;
    return BDDC_OK;
}

int bddc_host_setup_create(int n_instances, const bddc_instance* inst, const bddc_options* opt,
                           bddc_host_setup** out) {
    return host_setup_create(n_instances, inst, opt, out, nullptr);
}

int bddc_host_setup_create_gpu(int n_instances, const bddc_instance* inst, const bddc_options* opt,
                               bddc_host_setup** out) {
    return host_setup_create(n_instances, inst, opt, out, bddc::local_maps_device);
}

int bddc_host_setup_query(const bddc_host_setup* hs, const char* name, int64_t* count, int* elem_bytes) {
    if (!hs) return BDDC_E_INVALID_ARG;
    return export_named(hs->P, name, nullptr, count, elem_bytes) ? BDDC_OK : BDDC_E_INVALID_ARG;
}

int bddc_host_setup_copy(const bddc_host_setup* hs, const char* name, void* dst) {
    if (!hs || !dst) return BDDC_E_INVALID_ARG;
    return export_named(hs->P, name, dst, nullptr, nullptr) ? BDDC_OK : BDDC_E_INVALID_ARG;
}

void bddc_host_setup_destroy(bddc_host_setup* hs) { delete hs; }

}  // extern "C"

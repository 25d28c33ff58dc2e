// Sparse factorisation of the coarse problem (host, FP64).
//
// The coarse matrix of Algorithm 1 (Sec. 3: the saddle system over the
// coarse flux dofs W_Pi and one pressure per subdomain, plus the global-mean
// multiplier of a pure-flux problem) is a sum of subdomain element matrices
// [Psi^T S Psi, b; b^T 0].  Above a few thousand coarse dofs (3D partitions
// with thousands of subdomains) a dense inverse no longer fits, so the
// coarse problem is factored by a multifrontal method:
//   ordering   nested dissection over the subdomains: recursive bisection
//              of the subdomain centroids along the widest axis; the
//              separator of a split is the set of coarse dofs shared by
//              subdomains on both sides (coarse dofs of faces cut by the
//              plane; the pure-flux multiplier lands in the root).  The net
//              fluxes of the faces inside a face-connected set of
//              subdomains cancel in the sum of its pressure rows, so the
//              set's constant pressure mode is fixed only by faces outside it
//              (or by Dirichlet faces); eliminating it early would make a
//              pivot block singular.  So every node but the root passes one
//              subdomain pressure per connected component of its subtree up
//              to its parent, and keeps the others;
//   factor     per tree node, children first: the front [P, B] (P the
//              node's own dofs, B the dofs of ancestors it couples to) is
//              assembled from its subdomain elements (leaves) or its
//              children's update matrices, and partially factored:
//                X = F_PP^{-1},  H = X F_PB,  U = F_BB - F_BP H  (to the parent);
//   solve      forward, children first: t_P = b_P + (children's updates),
//              u_B = (children's updates) - H^T t_P;
//              backward, root first: x_P = X t_P - H x_B.
// The matrix is symmetric, so X and U are symmetrised and F_BP X = H^T.
// Each node keeps X (p x p) and H (p x q); the device solve in
// bddc_kernels.cu runs the same two sweeps level by level.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <thread>

#include "bddc_internal.hpp"
#include "dense.hpp"

namespace bddc {
namespace {

struct Builder {
    int n;
    const std::vector<CoarseElement>& el;
    const std::vector<char>& is_pressure;
    int leaf_max;
    std::vector<std::vector<int>> inc;  // dof -> elements touching it
    std::vector<int> owner;             // dof -> node (-1 free, -2 reserved)
    std::vector<int> side;              // element -> 0 / 1 in the current split
    CoarseFactor& f;
    std::vector<std::vector<int>> leaf_el;  // node -> its elements (leaves)

    Builder(int n_, const std::vector<CoarseElement>& el_, const std::vector<char>& isp, int leaf_max_,
            CoarseFactor& out)
        : n(n_), el(el_), is_pressure(isp), leaf_max(leaf_max_), inc(n_), owner(n_, -1), side(el_.size(), 0),
          f(out), comp(el_.size(), 0), mark(el_.size(), 0) {
        for (int s = 0; s < (int)el.size(); ++s)
            for (int d : el[s].dofs) inc[d].push_back(s);
    }

    int new_node(std::vector<int>&& piv, int c0, int c1, std::vector<int>&& els) {
        const int id = (int)f.piv.size();
        std::sort(piv.begin(), piv.end());
        for (int d : piv) owner[d] = id;
        f.piv.push_back(std::move(piv));
        f.child0.push_back(c0);
        f.child1.push_back(c1);
        f.parent.push_back(-1);
        if (c0 >= 0) f.parent[c0] = id;
        if (c1 >= 0) f.parent[c1] = id;
        leaf_el.push_back(std::move(els));
        return id;
    }

    std::vector<int> comp;  // element -> union-find parent (within the current subtree)
    std::vector<int> mark;  // element -> stamp of the current subtree
    int stamp = 0;

    int find(int a) {
        while (comp[a] != a) a = comp[a] = comp[comp[a]];
        return a;
    }

    // connected components of the elements subs, linked by the coarse dofs
    // two of them share (faces); returns the component root of each element
    void components(const std::vector<int>& subs) {
        ++stamp;
        for (int s : subs) {
            mark[s] = stamp;
            comp[s] = s;
        }
        for (int s : subs)
            for (int d : el[s].dofs)
                if (inc[d].size() == 2) {
                    const int t = inc[d][0] == s ? inc[d][1] : inc[d][0];
                    if (mark[t] != stamp) continue;
                    const int a = find(s), b = find(t);
                    if (a != b) comp[std::max(a, b)] = std::min(a, b);
                }
    }

    // of the pressure dofs cand (sorted), keep one per connected component of
    // subs to pass up (returned) and move the others into piv; at the root
    // every one goes into piv
    std::vector<int> defer(const std::vector<int>& subs, const std::vector<int>& cand, std::vector<int>& piv,
                           bool root) {
        std::vector<int> up;
        if (root) {
            piv.insert(piv.end(), cand.begin(), cand.end());
            return up;
        }
        components(subs);
        std::vector<int> taken;
        for (int d : cand) {
            const int r = find(inc[d][0]);
            if (std::find(taken.begin(), taken.end(), r) == taken.end()) {
                taken.push_back(r);
                up.push_back(d);
            } else {
                piv.push_back(d);
            }
        }
        return up;
    }

    // returns the node and the pressure dofs it passes to its parent
    std::pair<int, std::vector<int>> build(std::vector<int> subs, bool root) {
        if ((int)subs.size() <= leaf_max) {
            std::vector<int> piv, pres;
            for (int s : subs)
                for (int d : el[s].dofs)
                    if (owner[d] == -1) {
                        owner[d] = -2;
                        (is_pressure[d] ? pres : piv).push_back(d);
                    }
            std::sort(pres.begin(), pres.end());
            std::vector<int> up = defer(subs, pres, piv, root);
            return {new_node(std::move(piv), -1, -1, std::vector<int>(subs)), std::move(up)};
        }
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int s : subs)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], el[s].c[a]);
                hi[a] = std::max(hi[a], el[s].c[a]);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
        std::sort(subs.begin(), subs.end(), [&](int a, int b) {
            return el[a].c[ax] < el[b].c[ax] || (el[a].c[ax] == el[b].c[ax] && a < b);
        });
        const size_t mid = subs.size() / 2;
        for (size_t i = 0; i < subs.size(); ++i) side[subs[i]] = i < mid ? 0 : 1;
        // separator: free dofs touched from both sides (every element that
        // touches a free dof of this subtree belongs to it)
        std::vector<int> sep;
        for (size_t i = 0; i < mid; ++i)
            for (int d : el[subs[i]].dofs) {
                if (owner[d] != -1) continue;
                for (int t : inc[d])
                    if (side[t] == 1) {
                        owner[d] = -2;
                        sep.push_back(d);
                        break;
                    }
            }
        std::vector<int> L(subs.begin(), subs.begin() + mid), R(subs.begin() + mid, subs.end());
        auto [c0, u0] = build(std::move(L), false);
        auto [c1, u1] = build(std::move(R), false);
        std::vector<int> cand(u0);
        cand.insert(cand.end(), u1.begin(), u1.end());
        std::sort(cand.begin(), cand.end());
        std::vector<int> up = defer(subs, cand, sep, root);
        return {new_node(std::move(sep), c0, c1, {}), std::move(up)};
    }
};

void sorted_union(const std::vector<int>& a, const std::vector<int>& b, std::vector<int>& out) {
    out.clear();
    std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
}

}  // namespace

SetupResult factor_coarse(int n, const std::vector<CoarseElement>& el, const std::vector<char>& is_pressure,
                          int leaf_max, int nthreads, CoarseFactor& f) {
    f = CoarseFactor();
    f.n = n;
    if (n <= 0 || el.empty() || (int)is_pressure.size() != n) return {BDDC_E_SETUP, "empty coarse problem"};
    Builder B(n, el, is_pressure, std::max(1, leaf_max), f);
    {
        std::vector<int> all(el.size());
        std::iota(all.begin(), all.end(), 0);
        f.root = B.build(std::move(all), true).first;
    }
    for (int d = 0; d < n; ++d)
        if (B.owner[d] < 0) return {BDDC_E_SETUP, "coarse dof not reached by the dissection"};
    const int nn = (int)f.piv.size();
    // depth (root 0) and boundary sets, children first (creation order)
    f.depth.assign(nn, 0);
    for (int v = nn - 1; v >= 0; --v)
        if (f.parent[v] >= 0) f.depth[v] = f.depth[f.parent[v]] + 1;
    f.max_depth = *std::max_element(f.depth.begin(), f.depth.end());
    f.bnd.assign(nn, {});
    for (int v = 0; v < nn; ++v) {
        std::vector<int> s;
        if (f.child0[v] < 0) {
            for (int e : B.leaf_el[v])
                for (int d : el[e].dofs) s.push_back(d);
            std::sort(s.begin(), s.end());
            s.erase(std::unique(s.begin(), s.end()), s.end());
        } else {
            sorted_union(f.bnd[f.child0[v]], f.bnd[f.child1[v]], s);
        }
        std::vector<int> b;
        std::set_difference(s.begin(), s.end(), f.piv[v].begin(), f.piv[v].end(), std::back_inserter(b));
        f.bnd[v] = std::move(b);
    }
    f.X.assign(nn, {});
    f.H.assign(nn, {});
    std::vector<std::vector<double>> U(nn);
    std::vector<SetupResult> res(nn);
    // numeric factorisation, deepest level first; nodes of a level in parallel
    for (int lev = f.max_depth; lev >= 0; --lev) {
        std::vector<int> nodes;
        for (int v = 0; v < nn; ++v)
            if (f.depth[v] == lev) nodes.push_back(v);
        std::atomic<size_t> next(0);
        auto work = [&]() {
            std::vector<int> pos(n, -1);
            for (size_t it; (it = next.fetch_add(1)) < nodes.size();) {
                const int v = nodes[it];
                const std::vector<int>& P = f.piv[v];
                const std::vector<int>& Bd = f.bnd[v];
                const int p = (int)P.size(), q = (int)Bd.size(), fs = p + q;
                for (int i = 0; i < p; ++i) pos[P[i]] = i;
                for (int j = 0; j < q; ++j) pos[Bd[j]] = p + j;
                std::vector<double> F((size_t)fs * fs, 0.0);
                if (f.child0[v] < 0) {
                    for (int e : B.leaf_el[v]) {
                        const CoarseElement& E = el[e];
                        const int m = (int)E.dofs.size();
                        for (int a = 0; a < m; ++a) {
                            const size_t ra = (size_t)pos[E.dofs[a]] * fs;
                            for (int b = 0; b < m; ++b) F[ra + pos[E.dofs[b]]] += E.E[(size_t)a * m + b];
                        }
                    }
                } else {
                    for (int c : {f.child0[v], f.child1[v]}) {
                        const std::vector<int>& cb = f.bnd[c];
                        const int qc = (int)cb.size();
                        for (int a = 0; a < qc; ++a) {
                            const size_t ra = (size_t)pos[cb[a]] * fs;
                            for (int b = 0; b < qc; ++b) F[ra + pos[cb[b]]] += U[c][(size_t)a * qc + b];
                        }
                        std::vector<double>().swap(U[c]);
                    }
                }
                std::vector<double> Fpp((size_t)p * p), Hm((size_t)p * q), X((size_t)p * p, 0.0);
                for (int i = 0; i < p; ++i)
                    for (int k = 0; k < p; ++k) Fpp[(size_t)i * p + k] = F[(size_t)i * fs + k];
                for (int i = 0; i < p; ++i)
                    for (int j = 0; j < q; ++j) Hm[(size_t)i * q + j] = F[(size_t)i * fs + p + j];
                std::vector<int> piv;
                if (p > 0) {
                    if (!lu(p, Fpp.data(), piv)) {
                        res[v] = {BDDC_E_SETUP, "singular pivot block in the coarse factorisation"};
                    } else {
                        for (int i = 0; i < p; ++i) X[(size_t)i * p + i] = 1.0;
                        lu_solve(p, Fpp.data(), piv, X.data(), p);
                        if (q > 0) lu_solve(p, Fpp.data(), piv, Hm.data(), q);
                        for (int i = 0; i < p; ++i)
                            for (int k = i + 1; k < p; ++k) {
                                const double s = 0.5 * (X[(size_t)i * p + k] + X[(size_t)k * p + i]);
                                X[(size_t)i * p + k] = s;
                                X[(size_t)k * p + i] = s;
                            }
                    }
                }
                // update matrix for the parent: U = F_BB - F_BP H
                std::vector<double> Uv((size_t)q * q);
                for (int a = 0; a < q; ++a) {
                    double* ua = Uv.data() + (size_t)a * q;
                    for (int b = 0; b < q; ++b) ua[b] = F[(size_t)(p + a) * fs + p + b];
                    for (int k = 0; k < p; ++k) {
                        const double l = F[(size_t)(p + a) * fs + k];
                        if (l == 0.0) continue;
                        const double* hk = Hm.data() + (size_t)k * q;
                        for (int b = 0; b < q; ++b) ua[b] -= l * hk[b];
                    }
                }
                for (int a = 0; a < q; ++a)
                    for (int b = a + 1; b < q; ++b) {
                        const double s = 0.5 * (Uv[(size_t)a * q + b] + Uv[(size_t)b * q + a]);
                        Uv[(size_t)a * q + b] = s;
                        Uv[(size_t)b * q + a] = s;
                    }
                for (double x : X)
                    if (!std::isfinite(x)) res[v] = {BDDC_E_SETUP, "non-finite coarse factor"};
                for (double x : Hm)
                    if (!std::isfinite(x)) res[v] = {BDDC_E_SETUP, "non-finite coarse factor"};
                f.X[v] = std::move(X);
                f.H[v] = std::move(Hm);
                U[v] = std::move(Uv);
                for (int d : P) pos[d] = -1;
                for (int d : Bd) pos[d] = -1;
            }
        };
        const int nt = (int)std::max<size_t>(1, std::min<size_t>(std::max(1, nthreads), nodes.size()));
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work);
        work();
        for (auto& t : th) t.join();
        for (int v : nodes)
            if (res[v].code) return res[v];
    }
    return {};
}

void coarse_factor_solve(const CoarseFactor& f, const double* b, double* x) {
    const int nn = (int)f.piv.size();
    std::vector<std::vector<double>> u(nn);
    std::vector<double> t(f.n, 0.0);
    // the update a child passes for dof d (0 if d is not in its boundary)
    auto from_child = [&](int c, int d) -> double {
        if (c < 0) return 0.0;
        const std::vector<int>& cb = f.bnd[c];
        const auto it = std::lower_bound(cb.begin(), cb.end(), d);
        return (it != cb.end() && *it == d) ? u[c][it - cb.begin()] : 0.0;
    };
    for (int v = 0; v < nn; ++v) {
        const std::vector<int>& P = f.piv[v];
        const std::vector<int>& Bd = f.bnd[v];
        const int p = (int)P.size(), q = (int)Bd.size();
        for (int i = 0; i < p; ++i) t[P[i]] = b[P[i]] + from_child(f.child0[v], P[i]) + from_child(f.child1[v], P[i]);
        u[v].assign(q, 0.0);
        for (int j = 0; j < q; ++j) {
            double acc = 0.0;
            for (int i = 0; i < p; ++i) acc += f.H[v][(size_t)i * q + j] * t[P[i]];
            u[v][j] = from_child(f.child0[v], Bd[j]) + from_child(f.child1[v], Bd[j]) - acc;
        }
    }
    for (int v = nn - 1; v >= 0; --v) {
        const std::vector<int>& P = f.piv[v];
        const std::vector<int>& Bd = f.bnd[v];
        const int p = (int)P.size(), q = (int)Bd.size();
        for (int i = 0; i < p; ++i) {
            double acc = 0.0;
            for (int k = 0; k < p; ++k) acc += f.X[v][(size_t)k * p + i] * t[P[k]];
            for (int j = 0; j < q; ++j) acc -= f.H[v][(size_t)i * q + j] * x[Bd[j]];
            x[P[i]] = acc;
        }
    }
}

}  // namespace bddc

"""Pins of the oracle's BDDC method (Algorithms 1-3), CPU only.

Pinned against: the direct solve of the assembled system, the exact
constant-coefficient solution, invariants the paper states (balanced
preconditioner output, divergence-free correction, mass conservation of u*,
symmetry, E a projection), brute-force spectra of the preconditioned
operator, a textbook CG run for the Lanczos estimate, and the paper's printed
iteration counts and condition numbers for k = 1.
"""

import json
import os

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, \
    pressure_drop_bc
from oracle import BDDCOracle, direct_solve, lanczos_condition
from oracle.adaptive import adaptive_constraints
from oracle.discretization import residuals

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def c1():
    return BDDCOracle(make_config("c1"))


def _wells(pb, rate=2.0):
    pb.f = np.zeros(pb.grid.n_cells)
    pb.f[0] = rate / pb.grid.cell_volume
    pb.f[-1] = -rate / pb.grid.cell_volume
    return pb


def test_lanczos_estimate_of_textbook_cg():
    """Plain CG on diag(1..60): the Lanczos estimate of the converged run is
    the exact condition number 60."""
    rng = np.random.default_rng(0)
    d = np.arange(1.0, 61.0)
    b = rng.standard_normal(60)
    x = np.zeros(60)
    r = b.copy()
    p = r.copy()
    rho = r @ r
    al, be = [], []
    for _ in range(200):
        q = d * p
        a = rho / (p @ q)
        x += a * p
        r -= a * q
        al.append(a)
        rn = r @ r
        if np.sqrt(rn) < 1e-13 * np.linalg.norm(b):
            break
        be.append(rn / rho)
        p = r + (rn / rho) * p
        rho = rn
    assert abs(lanczos_condition(al, be) - 60.0) < 1e-6


@pytest.mark.parametrize("name", ["c1", "tiny3d"])
def test_matches_direct_solve(name):
    pb = make_config(name)
    o = BDDCOracle(pb)
    res = o.solve(tol=1e-12)
    fd, pd = direct_solve(o.disc)
    assert np.linalg.norm(res.flux - fd) <= 1e-10 * np.linalg.norm(fd)
    assert np.linalg.norm(res.pressure - pd) <= 1e-10 * np.linalg.norm(pd)


def test_pure_flux_wells_match_direct_solve_with_zero_mean_pressure():
    pb = _wells(make_config("c1"))
    t = pb.bc_type.copy()
    t[t == 1] = 0
    pb.bc_type, pb.bc_value = t, np.zeros_like(pb.bc_value)
    o = BDDCOracle(pb)
    res = o.solve(tol=1e-12)
    fd, pd = direct_solve(o.disc)
    assert np.linalg.norm(res.flux - fd) <= 1e-10 * np.linalg.norm(fd)
    assert abs(np.mean(res.pressure)) < 1e-10 * np.abs(pd).max()
    assert np.linalg.norm(res.pressure - pd) <= 1e-9 * np.linalg.norm(pd)


@pytest.mark.parametrize("part", ["regular", "irregular"])
def test_constant_k_closed_form_any_partition(part):
    g = Grid(2, (18, 12, 1), (1.0, 0.5, 1.0))
    p = box_partition(g, (3, 3)) if part == "regular" else irregular_box_partition(g, 3)
    t, v = pressure_drop_bc(g)
    k = 2.0
    o = BDDCOracle(Problem("cf", g, np.full(g.n_cells, k), p, t, v, np.zeros(g.n_cells)))
    res = o.solve(tol=1e-13)
    L = g.n[0] * g.h[0]
    nxf = (g.n[0] + 1) * g.n[1]
    area = g.h[1]
    assert np.allclose(res.flux[:nxf], k * area / L, rtol=1e-11, atol=0)
    assert np.allclose(res.flux[nxf:], 0.0, atol=1e-11 * k * area / L)
    xc = (np.arange(g.n_cells) % g.n[0] + 0.5) * g.h[0]
    assert np.allclose(res.pressure, 1.0 - xc / L, atol=1e-11)


def test_mass_conservation_and_divergence_free_correction():
    """u* from Steps 1-2 satisfies b(u*, q) = <f, q> for all q, and u_corr is
    divergence-free (Remark 'scaling'), whatever the CG tolerance."""
    pb = _wells(make_config("c1"))
    o = BDDCOracle(pb)
    res = o.solve(tol=1e-2)
    disc = o.disc
    for u in (res.u_star, res.flux):
        _, r2 = residuals(disc, u, np.zeros(disc.n_cells))
        assert np.max(np.abs(r2)) < 1e-11 * np.max(np.abs(disc.cell_rhs()))
    # Step 1: b(u_0, 1_i) = <f, 1_i> per subdomain
    for sub in o.ss.subs:
        b_u0 = np.ones(len(sub.cells)) @ sub.B @ res.u0[sub.faces]
        assert abs(b_u0 - np.sum(disc.cell_rhs()[sub.cells])) < 1e-11


def test_operator_is_energy_of_stokes_harmonic_extension(c1):
    """v^T S^i v = a(Hv, Hv) and S^i is positive definite (Sec. 3)."""
    rng = np.random.default_rng(1)
    for loc in c1.local:
        v = rng.standard_normal(loc.ng)
        Hv = loc.H @ v
        assert np.isclose(v @ loc.S @ v, Hv @ loc.A @ Hv, rtol=1e-11)
        assert np.linalg.eigvalsh(loc.S)[0] > 0


def test_preconditioner_symmetric_and_balanced(c1):
    """M is symmetric and its output lies in the balanced space (Sec. 3,
    W_hat_B; Lemma 3 of the cited nested BDDC paper)."""
    rng = np.random.default_rng(2)
    r1, r2 = rng.standard_normal((2, c1.ss.n_gamma))
    z1, _ = c1.precondition(r1)
    z2, _ = c1.precondition(r2)
    assert np.isclose(r1 @ z2, r2 @ z1, rtol=1e-10)
    assert r1 @ z1 > 0
    _, bz = c1.apply_operator(z1, np.zeros(c1.ss.N))
    assert np.max(np.abs(bz)) < 1e-11 * np.max(np.abs(z1))


def test_averaging_operator_is_a_projection(c1):
    rng = np.random.default_rng(3)
    parts = [rng.standard_normal(s.n_gamma) for s in c1.ss.subs]
    e1 = c1.assemble(parts, weighted=True)
    e2 = c1.assemble(c1.restrict(e1), weighted=True)
    assert np.allclose(e1, e2, rtol=1e-14, atol=1e-14)
    total = c1.assemble([s.weights for s in c1.ss.subs])
    assert np.allclose(total, 1.0)


def test_pressure_rescaling_does_not_change_the_iterates():
    """The block rescaling D (Sec. 4) changes only the pressure variables: the
    flux iterates are the same with and without it."""
    pb = make_config("c1")
    a = BDDCOracle(pb, pressure_scaling=True).solve(tol=1e-10)
    b = BDDCOracle(pb, pressure_scaling=False).solve(tol=1e-10)
    # identical iterates up to rounding: the first steps agree to rounding
    # (later ones drift apart as finite-precision CG does), the iteration
    # counts nearly agree and both runs reach the same solution
    assert abs(a.iterations - b.iterations) <= 2
    assert np.allclose(a.relres[:10], b.relres[:10], rtol=1e-11)
    assert np.allclose(a.alphas[:10], b.alphas[:10], rtol=1e-11)
    assert np.linalg.norm(a.flux - b.flux) <= 1e-10 * np.linalg.norm(a.flux)
    assert np.linalg.norm(a.pressure - b.pressure) <= 1e-9 * np.linalg.norm(a.pressure)


def _preconditioned_spectrum(o):
    """Exact eigenvalues of M S on the balanced subspace (brute force)."""
    n, N = o.ss.n_gamma, o.ss.N
    B0 = np.zeros((N, n))
    S = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        q, bu = o.apply_operator(e, np.zeros(N))
        S[:, j] = q
        B0[:, j] = bu
    _, s, Vt = np.linalg.svd(B0)
    rank = int(np.sum(s > 1e-12 * s[0])) if s.size else 0
    Q = Vt[rank:].T
    MSQ = np.column_stack([o.precondition(S @ Q[:, k])[0] for k in range(Q.shape[1])])
    ev = np.linalg.eigvals(Q.T @ MSQ)
    return np.sort(ev.real)


def test_lanczos_kappa_matches_brute_force_spectrum(c1):
    ev = _preconditioned_spectrum(c1)
    assert ev[0] > 0.999999  # BDDC: lambda_min >= 1
    kappa_exact = ev[-1] / ev[0]
    res = c1.solve(tol=1e-12)
    assert res.kappa <= kappa_exact * (1 + 1e-6)
    assert res.kappa >= 0.95 * kappa_exact


def test_adaptive_tiny_tau_makes_preconditioner_exact():
    """tau below every nonzero local eigenvalue constrains every face jump:
    W_tilde = W_hat, so kappa = 1; the coarse space then holds the whole
    interface space and Steps 1-2 already give the exact solution."""
    o = BDDCOracle(make_config("c1"), tau=1e-9)
    res = o.solve(tol=1e-10)
    assert res.iterations <= 1
    fd, _ = direct_solve(o.disc)
    assert np.linalg.norm(res.u_star - fd) <= 1e-11 * np.linalg.norm(fd)
    ev = _preconditioned_spectrum(o)
    assert ev[-1] / ev[0] < 1 + 1e-8


def test_adaptive_indicator_and_theory_bound():
    """omega-tilde <= tau after Algorithm 3, and kappa <= omega-tilde N_F^2
    (remark after eq. (indicator))."""
    pb = make_config("c1")
    for tau in (3.0, 10.0):
        o = BDDCOracle(pb, tau=tau)
        assert o.omega_tilde <= tau
        ev = _preconditioned_spectrum(o)
        nf = 4
        assert ev[-1] / ev[0] <= o.omega_tilde * nf ** 2
        assert o.solve(tol=1e-10).kappa <= tau * 1.5


def test_nonzero_local_eigenvalues_at_most_face_dofs_minus_constraints(c1):
    """(I - E) has rank |face| on the pair space and one face constraint
    removes one more direction (cf. Fig. 4: the last eigenvalues are 0)."""
    _, _, eigs = adaptive_constraints(c1, np.inf)
    for fidx, lam in eigs.items():
        f = len(c1.ss.faces[fidx]["dofs"])
        nz = int(np.sum(lam > 1e-10 * max(lam[0], 1e-300)))
        assert nz <= f - 1


def test_pair_eigenvalues_equal_face_reduced_problem(c1):
    """Independent route to the nonzero eigenvalues of
    eq. (eigenvalue-problem-local-matrix): minimising the pair energy for a
    given face jump delta gives delta^T T delta with
    T = (D S^{-1} D^T)^{-1}, D = [I/2, -I/2] on the face copies, so the
    eigenvalues solve S_F delta = lambda T delta on {face sum of delta = 0},
    S_F = S^i_FF + S^j_FF."""
    _, _, eigs = adaptive_constraints(c1, np.inf)
    ss = c1.ss
    for fidx, lam in eigs.items():
        fa = ss.faces[fidx]
        li, lj = c1.local[fa["i"]], c1.local[fa["j"]]
        gi = {int(e): k for k, e in enumerate(ss.subs[fa["i"]].gamma)}
        gj = {int(e): k for k, e in enumerate(ss.subs[fa["j"]].gamma)}
        pi = [gi[int(e)] for e in fa["dofs"]]
        pj = [gj[int(e)] for e in fa["dofs"]]
        Si_inv = np.linalg.inv(li.S)
        Sj_inv = np.linalg.inv(lj.S)
        T = np.linalg.inv(0.25 * (Si_inv[np.ix_(pi, pi)] + Sj_inv[np.ix_(pj, pj)]))
        SF = li.S[np.ix_(pi, pi)] + lj.S[np.ix_(pj, pj)]
        c = fa["rows"][0][:, None]
        Z = np.linalg.svd(c.T)[2][1:].T
        import scipy.linalg as sla
        red = np.sort(sla.eigh(Z.T @ SF @ Z, Z.T @ T @ Z, eigvals_only=True))[::-1]
        nz = lam[lam > 1e-10 * lam[0]]
        assert np.allclose(red[: len(nz)], nz, rtol=1e-8)


def test_table1_counts_regular_partitions():
    from oracle.discretization import Discretization
    from oracle.substructure import Substructuring
    for cfg, key in (("pin2d", "table1_regular_2d_Hh10"), ("pin3d", "table1_regular_3d_Hh10")):
        pb = make_config(cfg)
        ss = Substructuring(Discretization(pb), pb.partition, matrices=False)
        want = {k: v for k, v in GOLDEN[key].items() if k != "cite"}
        assert ss.counts() == want


def test_paper_pin_2d_homogeneous():
    """Table 2, k = 1, regular H/h = 10: it = 14, kappa = 3.980 (tol 1e-6).
    Readings: SPE10 cell size 20 x 10 ft, corner wells, Euclidean norm of
    the reduced residual."""
    want = GOLDEN["table2_k1_Hh10"]
    res = BDDCOracle(make_config("pin2d")).solve(tol=1e-6)
    assert abs(res.iterations - want["it"]) <= 1
    assert abs(res.kappa - want["kappa"]) <= 0.005 * want["kappa"]


def test_paper_pin_3d_homogeneous():
    """Table 5, k = 1, regular H/h = 10: it = 25, kappa = 17.099.  kappa is
    pinned to 0.5% (the oracle gives 17.083); the iteration count depends on
    the unstated stopping details and is held to +-2 (partial pin: the oracle
    takes 23).  About 80 s of CPU time."""
    want = GOLDEN["table5_k1_Hh10"]
    res = BDDCOracle(make_config("pin3d")).solve(tol=1e-6)
    assert abs(res.iterations - want["it"]) <= 2
    assert abs(res.kappa - want["kappa"]) <= 0.005 * want["kappa"]

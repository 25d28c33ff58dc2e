"""Pins of the oracle's stiffness scaling (Sec. 5, the jumps experiment;
Sec. 3, Remark "scaling"), CPU only.

Pinned against: the closed form the paper states for RT0 (stiffness scaling
equals rho-scaling, weights k_i^-1 / (k_i^-1 + k_j^-1) when k jumps across
the subdomain interfaces only), the invariants of E (a projection, weights
summing to one), the direct solve of the assembled system, the
conservation of u* that the Remark requires of the weights, the adaptive
indicator bounds, and the paper's observation that with interface-aligned
jumps the stiffness-scaled method converges like the homogeneous problem
while multiplicity scaling does not.
"""

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, \
    pressure_drop_bc, subdomain_constant
from oracle import BDDCOracle, direct_solve
from oracle.discretization import residuals


def _irregular3d():
    g = Grid(3, (11, 9, 7), (1.0, 2.0, 0.5))
    rng = np.random.default_rng(9)
    perm = 10 ** rng.normal(0, 1.0, (g.n_cells, 3))
    t, v = pressure_drop_bc(g)
    return Problem("irr3", g, perm, irregular_box_partition(g, 4), t, v, np.zeros(g.n_cells))


def _aligned(grid, parts, seed, n_comp=1):
    part = box_partition(grid, parts)
    t, v = pressure_drop_bc(grid)
    perm = subdomain_constant(part, seed, n_comp=n_comp)
    return Problem("aligned", grid, perm, part.astype(np.int32), t, v, np.zeros(grid.n_cells))


def _face_axis(ss, fa):
    return int(ss.disc.face_axis(int(fa["dofs"][0])))


@pytest.mark.parametrize("dim", [2, 3])
def test_stiffness_weights_are_rho_scaling_for_aligned_jumps(dim):
    """With k constant in each subdomain (diagonal, anisotropic), the weight
    of subdomain i on every dof of the face shared with j is
    k_i^-1 / (k_i^-1 + k_j^-1) for the face's normal axis a (Sec. 5: for RT0
    stiffness scaling is rho-scaling); pressure faces keep weight 1."""
    if dim == 2:
        g = Grid(2, (12, 9, 1), (2.0, 1.0, 1.0))
        pb = _aligned(g, (4, 3), 17, n_comp=2)
    else:
        g = Grid(3, (6, 6, 4), (1.0, 0.5, 2.0))
        pb = _aligned(g, (3, 2, 2), 18, n_comp=3)
    o = BDDCOracle(pb, scaling="stiffness")
    ss = o.ss
    kp = np.asarray(pb.perm)
    checked = 0
    for fa in ss.faces:
        if fa["kind"] != "F":
            for e in fa["dofs"]:
                sub = ss.subs[fa["i"]]
                assert sub.weights[list(sub.gamma).index(int(e))] == 1.0
            continue
        a = _face_axis(ss, fa)
        ci = ss.subs[fa["i"]].cells[0]
        cj = ss.subs[fa["j"]].cells[0]
        ri, rj = 1.0 / kp[ci, a], 1.0 / kp[cj, a]
        for side, r_own in ((fa["i"], ri), (fa["j"], rj)):
            sub = ss.subs[side]
            pos = [list(sub.gamma).index(int(e)) for e in fa["dofs"]]
            assert np.allclose(sub.weights[pos], r_own / (ri + rj), rtol=1e-13)
            checked += len(pos)
    assert checked > 0


@pytest.mark.parametrize("case", ["c1", "irregular3d"])
def test_stiffness_weights_constant_per_face_and_E_a_projection(case):
    """On fields whose jumps are not aligned with the subdomains the weights
    are still one value per face side (the Remark "scaling"), the two sides
    sum to one, and E is a projection (E^2 = E) with E 1 = 1."""
    pb = make_config("c1") if case == "c1" else _irregular3d()
    o = BDDCOracle(pb, scaling="stiffness")
    ss = o.ss
    for fa in ss.faces:
        if fa["kind"] != "F":
            continue
        wsum = np.zeros(len(fa["dofs"]))
        for side in (fa["i"], fa["j"]):
            sub = ss.subs[side]
            w = sub.weights[[list(sub.gamma).index(int(e)) for e in fa["dofs"]]]
            assert np.ptp(w) == 0.0
            assert 0.0 < w[0] < 1.0
            wsum += w
        assert np.allclose(wsum, 1.0, rtol=1e-15)
    # the weights are not the multiplicity ones on a heterogeneous field
    assert any(np.any(np.abs(s.weights - 0.5) > 1e-3) for s in ss.subs)
    rng = np.random.default_rng(3)
    parts = [rng.standard_normal(s.n_gamma) for s in ss.subs]
    e1 = o.assemble(parts, weighted=True)
    e2 = o.assemble(o.restrict(e1), weighted=True)
    assert np.allclose(e1, e2, rtol=1e-14, atol=1e-14)
    assert np.allclose(o.assemble([s.weights for s in ss.subs]), 1.0)


@pytest.mark.parametrize("case", ["c1", "tiny3d", "irregular3d"])
@pytest.mark.parametrize("tau", [None, 4.0])
def test_stiffness_scaling_matches_direct_solve(case, tau):
    """Stiffness-scaled BDDC at tol 1e-12 reaches the solution of the
    assembled saddle system (<= 1e-10), and u* from Steps 1-2 is cellwise
    conservative (the property the Remark "scaling" ties to the weights)."""
    pb = {"c1": lambda: make_config("c1"), "tiny3d": lambda: make_config("tiny3d"),
          "irregular3d": _irregular3d}[case]()
    o = BDDCOracle(pb, tau=tau, scaling="stiffness")
    res = o.solve(tol=1e-12)
    fd, pd = direct_solve(o.disc)
    assert np.linalg.norm(res.flux - fd) <= 1e-10 * np.linalg.norm(fd)
    assert np.linalg.norm(res.pressure - pd) <= 1e-10 * np.linalg.norm(pd)
    _, r2 = residuals(o.disc, res.u_star, np.zeros(o.disc.n_cells))
    assert np.abs(r2).max() <= 1e-12 * max(1.0, np.abs(o.disc.cell_rhs()).max())
    if tau is not None:
        # Algorithm 3 with the stiffness weights in (I - E): omega-tilde <= tau
        assert o.omega_tilde <= tau


def test_stiffness_preconditioner_symmetric_and_balanced():
    """M with stiffness weights is symmetric, positive on a random residual
    and its output balanced (Sec. 3), as with multiplicity weights."""
    o = BDDCOracle(_irregular3d(), tau=4.0, scaling="stiffness")
    rng = np.random.default_rng(2)
    r1, r2 = rng.standard_normal((2, o.ss.n_gamma))
    z1, _ = o.precondition(r1)
    z2, _ = o.precondition(r2)
    assert np.isclose(r1 @ z2, r2 @ z1, rtol=1e-10)
    assert r1 @ z1 > 0
    _, bz = o.apply_operator(z1, np.zeros(o.ss.N))
    assert np.max(np.abs(bz)) < 1e-11 * np.max(np.abs(z1))


def test_interface_aligned_jumps_stiffness_converges_like_homogeneous():
    """Sec. 5, the jumps experiment: with k jumping by up to 1e6 across the
    interfaces only, stiffness-scaled BDDC converges like the k = 1 problem
    (the paper: kappa 4.046 with jumps against 4.050 with k = 1 on the same
    partition), while multiplicity scaling degrades by orders of magnitude.
    Geometry of the paper's 2D pins: 60 x 220 cells of 20 x 10 ft, 6 x 22
    subdomains, corner wells, tol 1e-6."""
    base = make_config("pin2d")
    ref = BDDCOracle(base).solve(tol=1e-6)
    pb = make_config("pin2d")
    pb.perm = subdomain_constant(pb.partition, 1045)
    st = BDDCOracle(pb, scaling="stiffness").solve(tol=1e-6)
    assert st.iterations <= ref.iterations + 2
    assert st.kappa <= 1.25 * ref.kappa
    mu = BDDCOracle(pb, scaling="multiplicity").solve(tol=1e-6, maxit=60)
    assert mu.kappa > 100.0 * st.kappa

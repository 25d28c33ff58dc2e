"""Pins of the oracle's MsMFEM constraints (Sec. 5, the comparison method)
and of its explicit constraint rows, CPU only.

Pinned against: a closed form of the pair problem on four cells (derived by
hand from the RT0 energy and mass balance), cellwise conservation and the
unit net flux of every pair solution, symmetry, minimal energy among
conservative fluxes, the well-weighted source distribution, the direct
solve of the assembled system, and the paper's two findings on these
constraints (a slight improvement over the initial constraints; adaptive
constraints of a coarse space no larger do much better).
"""

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, pressure_drop_bc
from oracle import BDDCOracle, direct_solve
from oracle.msmfem import pair_flux, msmfem_constraints


def _pair_2x2(k_bottom, k_top):
    """2 x 2 unit cells, subdomain 0 = left column, 1 = right column."""
    g = Grid(2, (2, 2, 1), (1.0, 1.0, 1.0))
    perm = np.array([k_bottom, k_bottom, k_top, k_top])
    t, v = pressure_drop_bc(g)
    part = np.array([0, 1, 0, 1], dtype=np.int32)
    return Problem("pair", g, perm, part, t, v, np.zeros(4))


@pytest.mark.parametrize("kb,kt", [(1.0, 1.0), (1.0, 7.0), (30.0, 0.2)])
def test_pair_flux_closed_form_four_cells(kb, kt):
    """Unit flow from the left column to the right one, no flow elsewhere:
    mass balance leaves one circulation v0 through the vertical faces, and
    minimising the RT0 energy (1/3 on the diagonal per face) gives
    v0 = (k_t - k_b) / (4 (k_t + k_b)), so the bottom face carries
    (k_t + 3 k_b) / (4 (k_t + k_b)) and the top one (3 k_t + k_b) / (4 (k_t + k_b))."""
    o = BDDCOracle(_pair_2x2(kb, kt), constraints="msmfem")
    face = [f for f in o.ss.faces if f["kind"] == "F"][0]
    row, _ = pair_flux(o, face)
    dofs = list(face["dofs"])  # the bottom x-face has the smaller id
    s = kt + kb
    assert np.allclose(row, [(kt + 3 * kb) / (4 * s), (3 * kt + kb) / (4 * s)], rtol=1e-13)


@pytest.mark.parametrize("name", ["c1", "tiny3d"])
def test_pair_solutions_are_conservative_with_unit_net_flux(name):
    """Every pair problem: div u = w_i on Omega^i and -w_j on Omega^j in
    every cell (exact), net flux 1 from i to j through the face."""
    o = BDDCOracle(make_config(name), constraints="msmfem")
    disc, ss = o.disc, o.ss
    for face in ss.faces:
        if face["kind"] != "F":
            continue
        row, (faces, u, cells, _) = pair_flux(o, face)
        _, B = disc.assemble(cells, faces)
        ni = len(ss.subs[face["i"]].cells)
        w = np.concatenate([np.full(ni, 1.0 / (ni * disc.vol)),
                            np.full(len(cells) - ni, -1.0 / ((len(cells) - ni) * disc.vol))])
        assert np.allclose(B @ u, -w * disc.vol, atol=1e-12)
        assert np.isclose(face["coef"] @ row, 1.0, rtol=1e-12)


def test_pair_flux_is_symmetric_and_energy_minimal():
    """A pair mirror-symmetric about the face's midline gives a symmetric
    face flux; adding a circulation (a divergence-free flux around an inner
    vertex) to the pair solution raises its energy."""
    g = Grid(2, (6, 4, 1), (1.0, 1.0, 1.0))
    rng = np.random.default_rng(4)
    k = 10 ** rng.normal(0, 1, (4, 6))
    k = 0.5 * (k + k[::-1])  # symmetric in y
    t, v = pressure_drop_bc(g)
    part = (np.arange(24) % 6 >= 3).astype(np.int32)
    o = BDDCOracle(Problem("sym", g, k.reshape(-1), part, t, v, np.zeros(24)), constraints="msmfem")
    face = [f for f in o.ss.faces if f["kind"] == "F"][0]
    row, (faces, u, cells, _) = pair_flux(o, face)
    assert np.allclose(row, row[::-1], rtol=1e-12)
    A, B = o.disc.assemble(cells, faces)
    # circulation around the vertex shared by cells (1,1), (2,1), (1,2), (2,2)
    pos = {int(e): n for n, e in enumerate(faces)}
    dz = np.zeros(len(faces))
    for e, sgn in ((o.disc.face_id(0, 2, 1, 0), 1.0), (o.disc.face_id(1, 2, 2, 0), 1.0),
                   (o.disc.face_id(0, 2, 2, 0), -1.0), (o.disc.face_id(1, 1, 2, 0), -1.0)):
        dz[pos[int(e)]] = sgn
    assert np.allclose(B @ dz, 0.0)
    e0 = u @ A @ u
    for eps in (1e-3, -1e-3, 0.1):
        uu = u + eps * dz
        assert uu @ A @ uu > e0


def test_pair_source_follows_the_well():
    """A subdomain with sources gets w = f / int f (Sec. 5): the pair
    solution's divergence follows the well's cells."""
    pb = make_config("c1")
    pb.f = np.zeros(pb.grid.n_cells)
    pb.f[0] = 3.0 / pb.grid.cell_volume
    pb.f[1] = 1.0 / pb.grid.cell_volume
    o = BDDCOracle(pb, constraints="msmfem")
    face = [f for f in o.ss.faces if f["kind"] == "F" and f["i"] == o.ss.part[0]][0]
    _, (faces, u, cells, _) = pair_flux(o, face)
    _, B = o.disc.assemble(cells, faces)
    div = -(B @ u) / o.disc.vol  # source density in each cell
    ci = list(cells)
    assert np.isclose(div[ci.index(0)], 0.75 / o.disc.vol, rtol=1e-12)
    assert np.isclose(div[ci.index(1)], 0.25 / o.disc.vol, rtol=1e-12)
    others = [n for n, c in enumerate(cells) if o.ss.part[c] == o.ss.part[0] and c not in (0, 1)]
    assert np.allclose(div[others], 0.0, atol=1e-12)


@pytest.mark.parametrize("name", ["c1", "tiny3d"])
def test_msmfem_bddc_matches_direct_solve(name):
    o = BDDCOracle(make_config(name), constraints="msmfem")
    res = o.solve(tol=1e-12)
    fd, pd = direct_solve(o.disc)
    assert np.linalg.norm(res.flux - fd) <= 1e-10 * np.linalg.norm(fd)
    assert np.linalg.norm(res.pressure - pd) <= 1e-10 * np.linalg.norm(pd)
    # one row per face between two subdomains (none is a multiple of the net-flux row here)
    n_faces = sum(1 for f in o.ss.faces if f["kind"] == "F")
    assert o.n_added == n_faces


@pytest.mark.parametrize("name", ["c1", "tiny3d"])
def test_paper_findings_on_msmfem_constraints(name):
    """Sec. 5: the multiscale constraints improve on the initial ones only
    slightly, and the adaptive constraints outperform them: with tau = 10
    the adaptive coarse space is no larger, and kappa is far smaller."""
    pb = make_config(name)
    face = BDDCOracle(pb).solve(tol=1e-10)
    ms = BDDCOracle(pb, constraints="msmfem")
    rms = ms.solve(tol=1e-10)
    ad = BDDCOracle(pb, tau=10.0)
    rad = ad.solve(tol=1e-10)
    assert rms.kappa < face.kappa
    assert ad.n_coarse <= ms.n_coarse
    assert rad.kappa < 0.2 * rms.kappa


def test_explicit_rows_reproduce_msmfem_and_are_validated():
    """The explicit constraint mode: the MsMFEM rows given as caller rows
    (global face ids and coefficients) build the same coarse space and
    solution; a row spread over two faces is rejected."""
    pb = make_config("c1")
    ms = BDDCOracle(pb, constraints="msmfem")
    rows = []
    for face in ms.ss.faces:
        if face["kind"] == "F":
            rows.append((face["dofs"], face["rows"][1]))
    ex = BDDCOracle(pb, constraints="explicit", explicit_rows=rows)
    assert ex.n_coarse == ms.n_coarse
    a, b = ms.solve(tol=1e-12), ex.solve(tol=1e-12)
    # the same space; the rows are orthonormalised once more, so the
    # iterates agree up to rounding (CG at kappa ~ 1e2 can end a step apart)
    assert abs(a.iterations - b.iterations) <= 1
    # both at tol 1e-12, each within ~1e-11 of the direct solve
    assert np.linalg.norm(a.flux - b.flux) <= 1e-10 * np.linalg.norm(a.flux)
    f0, f1 = [f for f in ms.ss.faces if f["kind"] == "F"][:2]
    bad = (np.concatenate([f0["dofs"][:1], f1["dofs"][:1]]), np.ones(2))
    with pytest.raises(ValueError):
        BDDCOracle(pb, constraints="explicit", explicit_rows=[bad])

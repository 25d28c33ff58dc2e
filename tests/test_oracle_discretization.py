"""Pins of the oracle's RT0/P0 discretisation (CPU only).

Each test checks the oracle against something other than itself: a quadrature
of the RT0 basis functions, the exact solution of a constant-coefficient
pressure drop, the convergence to a smooth manufactured solution, and the
paper's degree-of-freedom counts.
"""

import json
import os

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, \
    no_flow_bc, pressure_drop_bc
from oracle.discretization import Discretization, direct_solve, residuals

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_mass_block_matches_quadrature_of_rt0_basis():
    """a(phi_lo, phi_lo), a(phi_lo, phi_hi) by Gauss quadrature of the RT0
    basis on a 3D box (Sec. 2, eq. (a))."""
    g = Grid(3, (1, 1, 1), (0.3, 0.7, 1.9))
    k = np.array([[2.5, 0.4, 7.0]])
    pb = Problem("q", g, k, np.zeros(1, np.int32), *no_flow_bc(g), np.zeros(1))
    disc = Discretization(pb)
    xg, wg = np.polynomial.legendre.leggauss(4)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    for a in range(3):
        area = g.cell_volume / g.h[a]
        lo = lambda xi: (1 - xi) / area  # noqa: E731
        hi = lambda xi: xi / area        # noqa: E731
        def integ(f1, f2):
            return g.cell_volume * np.sum(wg * f1(xg) * f2(xg)) / k[0, a]
        ref = np.array([[integ(lo, lo), integ(lo, hi)], [integ(hi, lo), integ(hi, hi)]])
        assert np.allclose(disc.cell_mass_block(0, a), ref, rtol=1e-14, atol=0)


def _const_k_problem(grid, part, k=3.7):
    t, v = pressure_drop_bc(grid, 1.0, 0.0)
    return Problem("cf", grid, np.full(grid.n_cells, k), part, t, v, np.zeros(grid.n_cells))


@pytest.mark.parametrize("dim", [2, 3])
def test_direct_solve_reproduces_linear_pressure_exactly(dim):
    """Constant k, p = 1 -> 0 across x: u = k/L per unit area, p linear; RT0/P0
    reproduce it exactly (flux per face = k * area / L, P0 = p at centres)."""
    if dim == 2:
        g = Grid(2, (12, 7, 1), (0.5, 2.0, 1.0))
    else:
        g = Grid(3, (6, 5, 4), (0.5, 1.0, 0.25))
    k = 3.7
    disc = Discretization(_const_k_problem(g, np.zeros(g.n_cells, np.int32), k))
    flux, p = direct_solve(disc)
    L = g.n[0] * g.h[0]
    area_x = g.cell_volume / g.h[0]
    nx_faces = (g.n[0] + 1) * g.n[1] * g.n[2]
    assert np.allclose(flux[:nx_faces], k * area_x / L, rtol=1e-12, atol=0)
    assert np.allclose(flux[nx_faces:], 0.0, atol=1e-12 * k * area_x / L)
    xc = (np.arange(g.n_cells) % g.n[0] + 0.5) * g.h[0]
    assert np.allclose(p, 1.0 - xc / L, rtol=0, atol=1e-12)


def test_manufactured_smooth_solution_converges():
    """p = cos(pi x) cos(pi y) on the unit square, k = 1, no flow: u = -grad p,
    f = div u = 2 pi^2 p.  Cell-centre pressure and face fluxes converge at
    second order on uniform grids; a wrong sign of f or of b would not."""
    errs = []
    for n in (8, 16, 32):
        g = Grid(2, (n, n, 1), (1 / n, 1 / n, 1.0))
        t, v = no_flow_bc(g)
        x = (np.arange(g.n_cells) % n + 0.5) / n
        y = (np.arange(g.n_cells) // n + 0.5) / n
        pex = np.cos(np.pi * x) * np.cos(np.pi * y)
        f = 2 * np.pi ** 2 * pex
        pb = Problem("m", g, np.ones(g.n_cells), np.zeros(g.n_cells, np.int32), t, v, f)
        disc = Discretization(pb)
        flux, p = direct_solve(disc)
        # exact x-face flux: int over the face of -dp/dx dy (face at x = i/n)
        i = np.arange(n + 1)[None, :]
        j = np.arange(n)[:, None]
        xf = i / n
        fx = (np.pi * np.sin(np.pi * xf) / np.pi) * (np.sin(np.pi * (j + 1) / n) - np.sin(np.pi * j / n))
        errs.append((np.max(np.abs(p - pex)), np.max(np.abs(flux[: (n + 1) * n] - fx.reshape(-1)))))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[:, 0] > 1.8), rates
    assert np.all(rates[:, 1] > 1.8), rates


def test_paper_dof_counts():
    """Sec. 5: 39,880 dofs per 2D layer and 110,700 for the 3D cutouts
    (all faces plus all cells)."""
    d2 = Discretization(make_config("pin2d"))
    d3 = Discretization(make_config("pin3d"))
    assert d2.n_faces + d2.n_cells == GOLDEN["dofs_2d_layer"]["dofs"]
    assert d3.n_faces + d3.n_cells == GOLDEN["dofs_3d_cutout"]["dofs"]


def test_wells_mass_balance_and_direct_residual():
    pb = make_config("c1")
    pb.f = np.zeros_like(pb.f)
    pb.f[0], pb.f[-1] = 5.0, -5.0
    disc = Discretization(pb)
    flux, p = direct_solve(disc)
    r1, r2 = residuals(disc, flux, p)
    assert np.max(np.abs(r1)) < 1e-10 and np.max(np.abs(r2)) < 1e-12


def test_irregular_partition_generator_is_a_box_partition():
    g = Grid(3, (17, 13, 11), (1, 1, 1))
    part = irregular_box_partition(g, 7)
    ids = np.unique(part)
    assert ids[0] == 0 and ids[-1] == len(ids) - 1
    p3 = part.reshape(11, 13, 17)
    for s in ids:
        kk, jj, ii = np.nonzero(p3 == s)
        box = (kk.max() - kk.min() + 1) * (jj.max() - jj.min() + 1) * (ii.max() - ii.min() + 1)
        assert box == len(kk)
        for ext in (np.ptp(kk) + 1, np.ptp(jj) + 1, np.ptp(ii) + 1):
            assert 3 <= ext <= 10
    assert np.array_equal(box_partition(g, (1, 1, 1)), np.zeros(g.n_cells, np.int32))

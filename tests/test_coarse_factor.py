"""The sparse coarse solver on the CPU (no GPU needed): the multifrontal
factor over a nested dissection of the subdomains (bddc_coarse.cpp) solves
the coarse problem of Algorithm 1 (Sec. 3, eqs. (two-level_coarse-1/2)) as
the dense inverse does, its dissection tree is a valid elimination
structure, and the whole method emulated with it matches the oracle."""

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, layered_3d, \
    pressure_drop_bc, no_flow_bc
from oracle import BDDCOracle
from paper_1901_02090_gb300 import bddc

from packed_emulation import Packed, emulate_solve
from parity import FP64_REL, iteration_slack


def _slab3d():
    g = Grid(3, (20, 40, 15), (20.0, 10.0, 2.0))
    t, v = pressure_drop_bc(g)
    return Problem("slab3d", g, layered_3d(g, 3085), box_partition(g, (4, 8, 3)).astype(np.int32), t, v,
                   np.zeros(g.n_cells))


def _irregular3d():
    g = Grid(3, (24, 20, 12), (20.0, 10.0, 2.0))
    t, v = pressure_drop_bc(g)
    return Problem("irr3d", g, layered_3d(g, 4085), irregular_box_partition(g, 4085).astype(np.int32), t, v,
                   np.zeros(g.n_cells))


def _pure_flux_2d():
    pb = make_config("pin2d")  # no-flow boundary, corner wells: the global-mean multiplier
    return pb


CASES = {"c1": lambda: make_config("c1"), "c2": lambda: make_config("c2"), "tiny3d": lambda: make_config("tiny3d"),
         "pin2d_pure_flux": _pure_flux_2d, "slab3d": _slab3d, "irregular3d": _irregular3d}


def _setups(pb, tau=10.0):
    dense = bddc.HostSetup([pb], bddc.default_options(tau=tau, coarse_solver=bddc.BDDC_COARSE_DENSE))
    sparse = bddc.HostSetup([pb], bddc.default_options(tau=tau, coarse_solver=bddc.BDDC_COARSE_SPARSE))
    return dense, sparse


@pytest.mark.parametrize("case", list(CASES))
def test_sparse_coarse_solve_matches_dense_inverse(case):
    dense, sparse = _setups(CASES[case]())
    ncn = int(dense.get("inst_ncn")[0])
    assert len(dense.get("cn_p")) == 0 and len(sparse.get("Kinv")) == 0
    rng = np.random.default_rng(7)
    for _ in range(3):
        b = rng.standard_normal(ncn)
        xd, xs = dense.coarse_solve(0, b), sparse.coarse_solve(0, b)
        assert np.linalg.norm(xs - xd) <= 1e-9 * np.linalg.norm(xd)
    dense.close()
    sparse.close()


@pytest.mark.parametrize("case", list(CASES))
def test_dissection_tree_is_an_elimination_structure(case):
    """Every coarse dof is eliminated by exactly one node; every entry of a
    child's update vector is consumed by exactly one front position of a node
    one level up; the root is the last node and has no boundary; a pure-flux
    problem's multiplier is eliminated at the root."""
    pb = CASES[case]()
    hs = bddc.HostSetup([pb], bddc.default_options(tau=10.0, coarse_solver=bddc.BDDC_COARSE_SPARSE))
    n = int(hs.get("inst_csoff")[1])
    p, q, depth = hs.get("cn_p"), hs.get("cn_q"), hs.get("cn_depth")
    od, ou = hs.get("cn_off_dof"), hs.get("cn_off_u")
    dof, c0, c1 = hs.get("cn_dof"), hs.get("cn_c0"), hs.get("cn_c1")
    nn = len(p)
    piv = np.concatenate([dof[od[v]:od[v] + p[v]] for v in range(nn)])
    assert np.array_equal(np.sort(piv), np.arange(n))
    assert depth[nn - 1] == 0 and q[nn - 1] == 0 and np.count_nonzero(depth == 0) == 1
    owner_of_u = np.concatenate([np.full(q[v], v) for v in range(nn)]).astype(int)
    used = np.zeros(len(owner_of_u), dtype=int)
    for v in range(nn):
        for arr in (c0, c1):
            refs = arr[od[v]:od[v] + p[v] + q[v]]
            refs = refs[refs >= 0]
            used[refs] += 1
            assert np.all(depth[owner_of_u[refs]] == depth[v] + 1)
            # the dof a child passes up is the dof at that front position
            pos = np.nonzero(arr[od[v]:od[v] + p[v] + q[v]] >= 0)[0]
            for k in pos:
                u = arr[od[v] + k]
                ch = owner_of_u[u]
                assert dof[od[ch] + p[ch] + (u - ou[ch])] == dof[od[v] + k]
    assert np.all(used == 1)
    if case == "pin2d_pure_flux":
        root = dof[od[nn - 1]:od[nn - 1] + p[nn - 1]]
        assert n - 1 in root and n == int(hs.get("inst_ncn")[0]) + 1
    hs.close()


@pytest.mark.parametrize("case", ["c2", "pin2d_pure_flux", "tiny3d"])
def test_emulated_solve_with_sparse_coarse_matches_oracle(case):
    pb = CASES[case]()
    if case == "pin2d_pure_flux":
        tau = None
    else:
        tau = 10.0
    hs = bddc.HostSetup([pb], bddc.default_options(tau=tau, coarse_solver=bddc.BDDC_COARSE_SPARSE))
    flux, pres, its, _, _ = emulate_solve(Packed(hs), pb.f, pb.bc_value, 1e-8)
    ref = BDDCOracle(pb, tau=tau).solve(tol=1e-8)
    assert abs(its - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    kap = max(1.0, ref.kappa)
    assert np.linalg.norm(flux - ref.flux) <= FP64_REL * kap * np.linalg.norm(ref.flux)
    assert np.linalg.norm(pres - ref.pressure) <= FP64_REL * kap * np.linalg.norm(ref.pressure)
    hs.close()

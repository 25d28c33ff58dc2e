"""CPU checks of the C-ABI library: exported symbols, error handling, and the
native host setup against the oracle (no GPU needed).

The host setup is read back through bddc_host_setup_* and replayed in NumPy
(tests/packed_emulation.py) with the same arithmetic as the GPU kernel; the
result must match the oracle.
"""

import ctypes as C
import os
import re

import numpy as np
import pytest

from synth import make_config
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, \
    pressure_drop_bc, no_flow_bc
from oracle import BDDCOracle, lanczos_condition
from paper_1901_02090_gb300 import bddc

from packed_emulation import Packed, emulate_solve
from parity import iteration_slack

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "bddc.h")).read()
    declared = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(bddc_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(bddc.lib, name), name
    assert declared == set(bddc.EXPORTED)


def _wells(pb):
    pb.f = np.zeros(pb.grid.n_cells)
    pb.f[3] = 2.0 / pb.grid.cell_volume
    pb.f[-7] = -2.0 / pb.grid.cell_volume
    return pb


def _pure_flux(pb):
    t, v = no_flow_bc(pb.grid)
    pb.bc_type, pb.bc_value = t, v
    return _wells(pb)


def test_interface_schur_and_correction_match_oracle():
    pb = make_config("tiny3d")
    hs = bddc.HostSetup([pb])
    o = BDDCOracle(pb)
    ng, offS, S = hs.get("sub_ng"), hs.get("off_S"), hs.get("S")
    offF, F = hs.get("off_F"), hs.get("F")
    for s, loc in enumerate(o.local):
        n = int(ng[s])
        Sn = S[offS[s]:offS[s] + n * n].reshape(n, n)
        assert np.allclose(Sn, loc.S, rtol=0, atol=1e-12 * np.abs(loc.S).max())
        Fo = np.column_stack([loc.delta_solve(np.eye(n)[:, j])[:n] for j in range(n)])
        Fn = F[offF[s]:offF[s] + n * n].reshape(n, n)
        assert np.allclose(Fn, Fo, rtol=0, atol=1e-11 * np.abs(Fo).max())
    assert np.allclose(hs.get("sub_d"), [sub.d for sub in o.ss.subs], rtol=1e-14)


CASES = {
    "c1": lambda: make_config("c1"),
    "c1_wells_pure_flux": lambda: _pure_flux(make_config("c1")),
    "tiny3d": lambda: make_config("tiny3d"),
    "irregular2d": lambda: _irregular2d(),
}


def _irregular2d():
    g = Grid(2, (23, 17, 1), (2.0, 1.0, 1.0))
    rng = np.random.default_rng(5)
    perm = 10 ** rng.normal(0, 1.5, g.n_cells)
    t, v = pressure_drop_bc(g, 2.0, -1.0)
    f = np.zeros(g.n_cells)
    f[40] = 0.3
    return Problem("irr", g, perm, irregular_box_partition(g, 11), t, v, f)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("tau", [None, 4.0])
def test_packed_emulation_matches_oracle(case, tau):
    pb = CASES[case]()
    hs = bddc.HostSetup([pb], bddc.default_options(tau=tau or 0.0))
    P = Packed(hs)
    o = BDDCOracle(pb, tau=tau)
    # tol 1e-8: iteration counts within one (within 3% once kappa > 1e3,
    # where two finite-precision CG runs drift apart after ~10 steps);
    # tol 1e-12: the solutions agree to ~1e-10
    _, _, its, al, be = emulate_solve(P, pb.f, pb.bc_value, 1e-8)
    r = o.solve(tol=1e-8)
    assert abs(int(its[0]) - r.iterations) <= iteration_slack(r.iterations, r.kappa)
    assert abs(lanczos_condition(al[0], be[0]) - r.kappa) <= 1e-2 * r.kappa
    flux, pres, _, _, _ = emulate_solve(P, pb.f, pb.bc_value, 1e-12)
    r = o.solve(tol=1e-12)
    assert np.linalg.norm(flux - r.flux) <= 1e-9 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-8 * np.linalg.norm(r.pressure)
    if tau is not None:
        assert np.isclose(hs.get("inst_omega")[0], o.omega_tilde, rtol=1e-8)
        assert int(hs.get("inst_ncn")[0]) == o.n_coarse


def test_batched_setup_packs_instances_independently():
    pbs = [make_config("c1"), _irregular2d(), make_config("c1", seed=7)]
    hs = bddc.HostSetup(pbs, bddc.default_options(tau=4.0))
    P = Packed(hs)
    f = np.concatenate([pb.f for pb in pbs])
    bc = np.concatenate([pb.bc_value for pb in pbs])
    flux, pres, its, _, _ = emulate_solve(P, f, bc, 1e-10)
    fo = np.cumsum([0] + [len(pb.bc_type) for pb in pbs])
    co = np.cumsum([0] + [pb.grid.n_cells for pb in pbs])
    for b, pb in enumerate(pbs):
        alone = bddc.HostSetup([pb], bddc.default_options(tau=4.0))
        fa, pa, ia, _, _ = emulate_solve(Packed(alone), pb.f, pb.bc_value, 1e-10)
        assert its[b] == ia[0]
        assert np.array_equal(flux[fo[b]:fo[b + 1]], fa)
        assert np.array_equal(pres[co[b]:co[b + 1]], pa)


def test_setup_rejects_invalid_inputs():
    pb = make_config("c1")
    bad = make_config("c1")
    bad.perm = bad.perm.copy()
    bad.perm[3] = -1.0
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([bad])
    assert e.value.code == bddc.BDDC_E_PERM
    bad = make_config("c1")
    part = bad.partition.copy()
    part[0] = part.max() + 2          # id gap -> empty subdomain
    bad.partition = part
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([bad])
    assert e.value.code == bddc.BDDC_E_PARTITION
    bad = make_config("c1")
    part = bad.partition.copy()
    part[0] = 15                      # cell 0 joins a far subdomain: disconnected
    bad.partition = part
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([bad])
    assert e.value.code == bddc.BDDC_E_PARTITION
    bad = make_config("c1")
    t = bad.bc_type.copy()
    t[np.nonzero(t == -1)[0][0]] = 1  # pressure on an interior face
    bad.bc_type = t
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([bad])
    assert e.value.code == bddc.BDDC_E_INVALID_ARG
    assert bddc.HostSetup([pb]) is not None


def test_setup_rejects_invalid_autotune_option_and_get_tuning_null():
    """bddc_options.autotune takes 0 or 1 (checked before any device work);
    bddc_get_tuning rejects a null handle."""
    o = bddc.default_options(autotune=2)
    with pytest.raises(bddc.BDDCError) as e:
        bddc.setup([make_config("c1")], o)
    assert e.value.code == bddc.BDDC_E_INVALID_ARG
    assert bddc.default_options().autotune == 0
    t = bddc.bddc_tuning()
    assert bddc.lib.bddc_get_tuning(None, C.byref(t)) == bddc.BDDC_E_INVALID_ARG


def test_setup_without_gpu_reports_cuda_error_not_crash():
    """bddc_setup needs a GPU; without one it returns BDDC_E_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bddc.BDDCError) as e:
        bddc.setup([make_config("c1")])
    assert e.value.code == bddc.BDDC_E_CUDA


def test_server_without_gpu_and_invalid_arguments():
    """The serving entry points validate their arguments on the host; without
    a GPU server creation returns BDDC_E_CUDA instead of starting threads."""
    import ctypes as C
    import torch
    lib = bddc.lib
    out = C.c_void_p()
    o = bddc.default_options()
    assert lib.bddc_server_create(C.byref(o), 0, 4, C.byref(out)) == bddc.BDDC_E_INVALID_ARG
    assert lib.bddc_server_create(C.byref(o), 1 << 30, 0, C.byref(out)) == bddc.BDDC_E_INVALID_ARG
    assert lib.bddc_server_create(C.byref(o), 1 << 30, 4, None) == bddc.BDDC_E_INVALID_ARG
    # the full-space operator form needs the FP64 path
    bad = bddc.default_options(formulation=bddc.BDDC_FORM_FULL, precision=bddc.BDDC_PREC_FP32)
    assert lib.bddc_server_create(C.byref(bad), 1 << 30, 4, C.byref(out)) == bddc.BDDC_E_INVALID_ARG
    t = C.c_uint64()
    assert lib.bddc_submit(None, None, None, None, 1e-8, C.byref(t)) == bddc.BDDC_E_INVALID_ARG
    assert lib.bddc_poll(None, 1, None, None, None, None, None) == bddc.BDDC_E_INVALID_ARG
    assert lib.bddc_wait(None, 1, 0.0) == bddc.BDDC_E_INVALID_ARG
    lib.bddc_server_destroy(None)
    if not torch.cuda.is_available():
        assert lib.bddc_server_create(C.byref(o), 1 << 30, 4, C.byref(out)) == bddc.BDDC_E_CUDA


@pytest.mark.parametrize("case", ["c1", "irregular2d", "c1_wells_pure_flux"])
def test_mixed_precision_emulation_keeps_balance_and_accuracy(case):
    """FP32 correction operator and coarse basis (the mixed path): with the
    per-face net-flux correction and the closing FP64 pressure correction the
    solution stays cellwise conservative and within 1e-6 of the oracle."""
    from oracle.discretization import residuals
    pb = CASES[case]()
    hs = bddc.HostSetup([pb], bddc.default_options(tau=4.0, precision=bddc.BDDC_PREC_FP32))
    flux, pres, its, _, _ = emulate_solve(Packed(hs), pb.f, pb.bc_value, 1e-8, mixed=True)
    o = BDDCOracle(pb, tau=4.0)
    r = o.solve(tol=1e-10)
    assert np.linalg.norm(flux - r.flux) <= 1e-6 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-6 * np.linalg.norm(r.pressure)
    _, r2 = residuals(o.disc, flux, pres)
    scale = np.abs(flux).max() + np.abs(o.disc.cell_rhs()).max()
    assert np.abs(r2).max() <= 1e-11 * scale


def test_setup_maps_are_accurate_at_high_contrast():
    """The local maps and the coarse basis are refined against the exact
    local operators: at contrast ~1e7 the native solve matches the direct
    solve of the assembled system to ~1e-10."""
    from oracle import direct_solve
    pb = make_config("c2")
    o = BDDCOracle(pb)
    fd, pd = direct_solve(o.disc)
    hs = bddc.HostSetup([pb], bddc.default_options(tau=10.0))
    flux, pres, _, _, _ = emulate_solve(Packed(hs), pb.f, pb.bc_value, 1e-12)
    assert np.linalg.norm(flux - fd) <= 1e-10 * np.linalg.norm(fd)
    assert np.linalg.norm(pres - pd) <= 1e-10 * np.linalg.norm(pd)


@pytest.mark.parametrize("precision", [0, 1])
def test_packed_setup_does_not_depend_on_thread_count(precision):
    """The setup packs the operator blocks and coarse inverses in parallel
    (one task per subdomain and instance, at offsets fixed before the copy):
    every exported array is bitwise the same for 1 and 8 host threads."""
    pbs = [make_config("c1"), CASES["irregular2d"](), CASES["tiny3d"]()]
    one = bddc.HostSetup(pbs, bddc.default_options(tau=4.0, precision=precision, n_threads=1))
    many = bddc.HostSetup(pbs, bddc.default_options(tau=4.0, precision=precision, n_threads=8))
    for name in ("S", "F", "P", "P64", "Gpre", "Gpost", "Kinv", "off_S", "off_F", "off_P", "off_Gpre",
                 "off_Gpost", "slot_g", "slot_w", "cslot_c", "inst_kinv_off"):
        a, b = one.get(name), many.get(name)
        assert a.dtype == b.dtype and np.array_equal(a, b), name


def test_incompatible_pure_flux_data_solve_the_compatible_part():
    """No pressure face and a net source: the bordered coarse problem removes
    the mean source; the flux equations converge and every cell's mass
    residual is the mean source per cell (what true_relres reports)."""
    from oracle.discretization import Discretization, residuals
    pb = make_config("c1")
    pb.bc_type, pb.bc_value = no_flow_bc(pb.grid)
    pb.f = np.zeros(pb.grid.n_cells)
    pb.f[3] = 2.0 / pb.grid.cell_volume
    hs = bddc.HostSetup([pb], bddc.default_options(tau=4.0))
    flux, pres, its, _, _ = emulate_solve(Packed(hs), pb.f, pb.bc_value, 1e-10)
    r1, r2 = residuals(Discretization(pb), flux, pres)
    assert np.abs(r1).max() <= 1e-9 * np.abs(flux).max()
    mean_source = pb.f.sum() * pb.grid.cell_volume / pb.grid.n_cells
    assert np.allclose(np.abs(r2), abs(mean_source), rtol=1e-8)


@pytest.mark.parametrize("case", ["c1", "irregular2d", "tiny3d"])
@pytest.mark.parametrize("tau", [None, 4.0])
def test_stiffness_scaling_setup_matches_oracle(case, tau):
    """BDDC_SCALING_STIFFNESS: the native weights equal the oracle's (one
    value per face side, Sec. 3 Remark "scaling"), and the packed setup,
    replayed with the kernel's arithmetic, matches the oracle's stiffness-
    scaled solve: iterations, kappa, omega-tilde and the adaptive coarse
    space (the w-weighted face eigenproblems), and the solution at tol
    1e-12."""
    pb = CASES[case]()
    opt = bddc.default_options(tau=tau or 0.0, scaling=bddc.BDDC_SCALING_STIFFNESS)
    hs = bddc.HostSetup([pb], opt)
    P = Packed(hs)
    o = BDDCOracle(pb, tau=tau, scaling="stiffness")
    off, w = hs.get("off_slot"), hs.get("slot_w")
    for s, sub in enumerate(o.ss.subs):
        assert np.allclose(w[off[s]:off[s + 1]], sub.weights, rtol=1e-13, atol=0)
    _, _, its, al, be = emulate_solve(P, pb.f, pb.bc_value, 1e-8)
    r = o.solve(tol=1e-8)
    assert abs(int(its[0]) - r.iterations) <= iteration_slack(r.iterations, r.kappa)
    assert abs(lanczos_condition(al[0], be[0]) - r.kappa) <= 1e-2 * r.kappa
    flux, pres, _, _, _ = emulate_solve(P, pb.f, pb.bc_value, 1e-12)
    r = o.solve(tol=1e-12)
    assert np.linalg.norm(flux - r.flux) <= 1e-9 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-8 * np.linalg.norm(r.pressure)
    if tau is not None:
        assert np.isclose(hs.get("inst_omega")[0], o.omega_tilde, rtol=1e-8)
        assert int(hs.get("inst_ncn")[0]) == o.n_coarse


def _source_free(pb):
    pb.f = np.zeros(pb.grid.n_cells)
    return pb


@pytest.mark.parametrize("case", ["c1", "irregular2d", "tiny3d"])
def test_msmfem_constraints_setup_matches_oracle(case):
    """BDDC_CONSTRAINTS_MSMFEM (Sec. 5): the native rows come from the pair
    problem condensed onto the face with the local maps (bordered by the
    net-flux row), the oracle's from the pair's full Darcy problem; both
    give the same coarse space and solve (source-free fields: the library's
    setup uses the uniform source distribution)."""
    pb = _source_free(CASES[case]())
    hs = bddc.HostSetup([pb], bddc.default_options(constraints=bddc.BDDC_CONSTRAINTS_MSMFEM))
    P = Packed(hs)
    o = BDDCOracle(pb, constraints="msmfem")
    assert int(hs.get("inst_ncn")[0]) == o.n_coarse
    _, _, its, al, be = emulate_solve(P, pb.f, pb.bc_value, 1e-8)
    r = o.solve(tol=1e-8)
    assert abs(int(its[0]) - r.iterations) <= iteration_slack(r.iterations, r.kappa)
    assert abs(lanczos_condition(al[0], be[0]) - r.kappa) <= 1e-2 * r.kappa
    flux, pres, _, _, _ = emulate_solve(P, pb.f, pb.bc_value, 1e-12)
    r = o.solve(tol=1e-12)
    assert np.linalg.norm(flux - r.flux) <= 1e-9 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-8 * np.linalg.norm(r.pressure)


def test_explicit_constraint_rows_setup_matches_oracle_and_rejects_bad_rows():
    """BDDC_CONSTRAINTS_EXPLICIT: caller rows (the oracle's MsMFEM rows and
    a random row on some faces) give the oracle's coarse space and solve; a
    row over the dofs of two faces is rejected with BDDC_E_INVALID_ARG."""
    pb = make_config("c1")
    ms = BDDCOracle(pb, constraints="msmfem")
    rng = np.random.default_rng(12)
    rows = []
    for k, face in enumerate(f for f in ms.ss.faces if f["kind"] == "F"):
        rows.append((face["dofs"], face["rows"][1]))
        if k % 3 == 0:
            rows.append((face["dofs"], rng.standard_normal(len(face["dofs"]))))
    pb.constraint_rows = rows
    hs = bddc.HostSetup([pb], bddc.default_options(constraints=bddc.BDDC_CONSTRAINTS_EXPLICIT))
    o = BDDCOracle(pb, constraints="explicit", explicit_rows=rows)
    assert int(hs.get("inst_ncn")[0]) == o.n_coarse
    flux, pres, _, _, _ = emulate_solve(Packed(hs), pb.f, pb.bc_value, 1e-12)
    r = o.solve(tol=1e-12)
    assert np.linalg.norm(flux - r.flux) <= 1e-9 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-8 * np.linalg.norm(r.pressure)
    f0, f1 = [f for f in ms.ss.faces if f["kind"] == "F"][:2]
    pb.constraint_rows = [(np.concatenate([f0["dofs"][:1], f1["dofs"][:1]]), np.ones(2))]
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([pb], bddc.default_options(constraints=bddc.BDDC_CONSTRAINTS_EXPLICIT))
    assert e.value.code == bddc.BDDC_E_INVALID_ARG

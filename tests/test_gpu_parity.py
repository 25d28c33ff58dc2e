"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Element-wise comparisons of flux and pressure on seeded inputs, iteration
counts and Lanczos estimates, the Step-3 operator and the BDDC
preconditioner on random vectors, batching (each instance's result is the
same alone and in a batch), host versus device buffers, and edge cases.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import make_config  # noqa: E402
from synth.problems import Grid, Problem, box_partition, irregular_box_partition, \
    no_flow_bc, pressure_drop_bc  # noqa: E402
from oracle import BDDCOracle  # noqa: E402
from parity import FP64_REL, MIXED_REL, converged_bound, iteration_slack  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bddc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc as b
    return b


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def gpu_solve(bddc, pbs, tol, tau=None, precision=0, device_io=True, maxit=5000, check=True, scaling=0):
    opt = bddc.default_options(tau=tau or 0.0, precision=precision, maxit=maxit, scaling=scaling)
    stream = torch.cuda.current_stream().cuda_stream
    h = bddc.setup(pbs, opt, stream=stream)
    f = np.concatenate([pb.f for pb in pbs])
    bc = np.concatenate([pb.bc_value for pb in pbs])
    nf, nc = len(bc), len(f)
    if device_io:
        flux = torch.empty(nf, dtype=torch.float64, device="cuda")
        pres = torch.empty(nc, dtype=torch.float64, device="cuda")
        its = torch.empty(len(pbs), dtype=torch.int32, device="cuda")
        rc = h.solve(_dev(f), _dev(bc), tol, flux, pres, its, check=check)
        torch.cuda.synchronize()
        out = flux.cpu().numpy(), pres.cpu().numpy(), its.cpu().numpy()
    else:
        flux = np.empty(nf)
        pres = np.empty(nc)
        its = np.empty(len(pbs), dtype=np.int32)
        rc = h.solve(f, bc, tol, flux, pres, its, check=check)
        out = flux, pres, its
    stats = [h.stats(i) for i in range(len(pbs))]
    h.close()
    return out + (stats, rc)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _wells(pb, pure_flux=False):
    pb.f = np.zeros(pb.grid.n_cells)
    pb.f[0] = 1.0 / pb.grid.cell_volume
    pb.f[-1] = -1.0 / pb.grid.cell_volume
    if pure_flux:
        pb.bc_type, pb.bc_value = no_flow_bc(pb.grid)
    return pb


def _irregular2d():
    g = Grid(2, (23, 17, 1), (2.0, 1.0, 1.0))
    rng = np.random.default_rng(5)
    perm = 10 ** rng.normal(0, 1.0, g.n_cells)
    t, v = pressure_drop_bc(g, 2.0, -1.0)
    return Problem("irr", g, perm, irregular_box_partition(g, 11), t, v, np.zeros(g.n_cells))


def _irregular3d():
    g = Grid(3, (11, 9, 7), (1.0, 2.0, 0.5))
    rng = np.random.default_rng(9)
    perm = 10 ** rng.normal(0, 1.0, (g.n_cells, 3))
    t, v = pressure_drop_bc(g)
    return Problem("irr3", g, perm, irregular_box_partition(g, 4), t, v, np.zeros(g.n_cells))


CASES = {
    "c1": lambda: make_config("c1"),
    "c1_wells_pure_flux": lambda: _wells(make_config("c1"), pure_flux=True),
    "tiny3d": lambda: make_config("tiny3d"),
    "irregular2d": _irregular2d,
    "irregular3d_anisotropic": _irregular3d,
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("tau", [None, 4.0])
def test_fp64_solve_matches_oracle(bddc, case, tau):
    pb = CASES[case]()
    o = BDDCOracle(pb, tau=tau)
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, tau)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= max(FP64_REL, 1e-8 * ref.kappa)
    assert _rel(pres, ref.pressure) <= max(FP64_REL, 1e-8 * ref.kappa)
    assert abs(st[0].kappa - ref.kappa) <= 0.02 * ref.kappa
    # both converged: agreement to ~1e-10
    ref = o.solve(tol=1e-12)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-12, tau)
    bound = converged_bound(o, ref)
    assert _rel(flux, ref.flux) <= bound
    assert _rel(pres, ref.pressure) <= bound
    if tau is not None:
        assert np.isclose(st[0].omega_tilde, o.omega_tilde, rtol=1e-8)
        assert st[0].n_coarse == o.n_coarse


@pytest.mark.parametrize("case", ["c1", "tiny3d", "irregular3d_anisotropic"])
@pytest.mark.parametrize("tau", [None, 4.0])
def test_stiffness_scaling_matches_oracle(bddc, case, tau):
    """BDDC_SCALING_STIFFNESS (weights of E per face side, Sec. 3 Remark
    "scaling" and Sec. 5): the FP64 path against the oracle's stiffness-
    scaled solve at tol 1e-8 and 1e-12, with omega-tilde and the coarse size
    of the w-weighted face eigenproblems; the mixed path within its bound."""
    pb = CASES[case]()
    o = BDDCOracle(pb, tau=tau, scaling="stiffness")
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, tau, scaling=bddc.BDDC_SCALING_STIFFNESS)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= max(FP64_REL, 1e-8 * ref.kappa)
    assert _rel(pres, ref.pressure) <= max(FP64_REL, 1e-8 * ref.kappa)
    assert abs(st[0].kappa - ref.kappa) <= 0.02 * ref.kappa
    if tau is not None:
        assert np.isclose(st[0].omega_tilde, o.omega_tilde, rtol=1e-8)
        assert st[0].n_coarse == o.n_coarse
    flux32, pres32, _, _, _ = gpu_solve(bddc, [pb], 1e-8, tau, precision=bddc.BDDC_PREC_FP32,
                                        scaling=bddc.BDDC_SCALING_STIFFNESS)
    assert _rel(flux32, ref.flux) <= MIXED_REL and _rel(pres32, ref.pressure) <= MIXED_REL
    ref = o.solve(tol=1e-12)
    flux, pres, _, _, _ = gpu_solve(bddc, [pb], 1e-12, tau, scaling=bddc.BDDC_SCALING_STIFFNESS)
    bound = converged_bound(o, ref)
    assert _rel(flux, ref.flux) <= bound
    assert _rel(pres, ref.pressure) <= bound


@pytest.mark.parametrize("field", ["channelized", "aligned_jumps"])
def test_stiffness_scaling_60x220(bddc, field):
    """The 60 x 220 grid (6 x 22 subdomains) with stiffness scaling, both
    precisions, adaptive tau = 10: the channelized field (jumps across and
    along the interfaces) and a field constant per subdomain (jumps aligned
    with the interfaces, up to 1e6, the paper's stiffness-scaling case)."""
    from synth.problems import subdomain_constant
    from oracle.discretization import residuals
    pb = make_config("c2", seed=2093)
    if field == "aligned_jumps":
        pb.perm = subdomain_constant(pb.partition, 1045)
    o = BDDCOracle(pb, tau=10.0, scaling="stiffness")
    ref = o.solve(tol=1e-8)
    S = bddc.BDDC_SCALING_STIFFNESS
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, 10.0, scaling=S)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    assert np.isclose(st[0].omega_tilde, o.omega_tilde, rtol=1e-8)
    assert st[0].n_coarse == o.n_coarse
    flux32, pres32, _, _, _ = gpu_solve(bddc, [pb], 1e-8, 10.0, precision=bddc.BDDC_PREC_FP32, scaling=S)
    assert _rel(flux32, ref.flux) <= MIXED_REL and _rel(pres32, ref.pressure) <= MIXED_REL
    for u, p_ in ((flux, pres), (flux32, pres32)):
        _, r2 = residuals(o.disc, u, p_)
        assert np.abs(r2).max() <= 1e-10 * np.abs(u).max()


@pytest.mark.parametrize("tau,seed", [(10.0, 2090), (100.0, 2090), (10.0, 2136)])
def test_channelized_60x220_fp64_and_fp32(bddc, tau, seed):
    """The 2D 60 x 220 channelized workload (6 x 22 subdomains, contrast ~1e7)
    at full size: FP64 path within 1e-8 of the oracle, FP32-apply path within
    1e-6 after the FP64 CG converges to 1e-8, both cellwise conservative."""
    from oracle.discretization import residuals
    pb = make_config("c2", seed=seed)
    o = BDDCOracle(pb, tau=tau)
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, tau, precision=bddc.BDDC_PREC_FP64)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    # two solutions with relative residual 1e-8 differ by up to ~kappa * 1e-8
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    assert abs(st[0].kappa - ref.kappa) <= 0.02 * ref.kappa
    flux32, pres32, its32, st32, _ = gpu_solve(bddc, [pb], 1e-8, tau, precision=bddc.BDDC_PREC_FP32)
    assert _rel(flux32, ref.flux) <= MIXED_REL
    assert _rel(pres32, ref.pressure) <= MIXED_REL
    for u, p_ in ((flux, pres), (flux32, pres32)):
        _, r2 = residuals(o.disc, u, p_)
        assert np.abs(r2).max() <= 1e-10 * np.abs(u).max()
    # the FP32 preconditioner changes the iteration count (stated, not +-1)
    assert abs(int(its32[0]) - ref.iterations) <= 2 + int(0.25 * ref.iterations)
    # converged: FP64 path within the converged bound of the oracle
    ref = o.solve(tol=1e-12)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-12, tau, precision=bddc.BDDC_PREC_FP64)
    bound = converged_bound(o, ref)
    assert _rel(flux, ref.flux) <= bound
    assert _rel(pres, ref.pressure) <= bound


@pytest.mark.parametrize("pure_flux", [False, True])
def test_channelized_60x220_sources_both_precisions(bddc, pure_flux):
    """Corner wells on the 60 x 220 channelized field (sources in two
    subdomains, none elsewhere, so both the source and the source-free form
    of Step 2 and of the post-correction run in one solve): FP64 and FP32-apply
    paths against the oracle, cellwise conservative."""
    from oracle.discretization import residuals
    pb = _wells(make_config("c2", seed=2091), pure_flux=pure_flux)
    assert np.count_nonzero(pb.f) == 2
    o = BDDCOracle(pb, tau=10.0)
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, 10.0, precision=bddc.BDDC_PREC_FP64)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    flux32, pres32, its32, st32, _ = gpu_solve(bddc, [pb], 1e-8, 10.0, precision=bddc.BDDC_PREC_FP32)
    assert _rel(flux32, ref.flux) <= MIXED_REL
    assert _rel(pres32, ref.pressure) <= MIXED_REL
    for u, p_ in ((flux, pres), (flux32, pres32)):
        r1, r2 = residuals(o.disc, u, p_)
        assert np.abs(r2).max() <= 1e-10 * np.abs(u).max()


@pytest.mark.parametrize("tau", [10.0, 100.0])
def test_3d_subdomains_of_5_cubed_both_precisions(bddc, tau):
    """Subdomains shaped like the 60 x 220 x 85 workload's (5^3 cells, up to
    150 interface dofs: interior subdomains have six faces) on its 3D field
    generator (ln k = 2.5 x Gaussian with channel layers at the bottom),
    20 x 20 x 15 cells of 20 x 10 x 2 ft, 4 x 4 x 3 subdomains, adaptive
    constraints (face averages alone leave kappa ~ 1.6e5 on this field)."""
    from synth.problems import layered_3d
    g = Grid(3, (20, 20, 15), (20.0, 10.0, 2.0))
    t, v = pressure_drop_bc(g)
    pb = Problem("c3-shaped", g, layered_3d(g, 1901), box_partition(g, (4, 4, 3)), t, v, np.zeros(g.n_cells))
    o = BDDCOracle(pb, tau=tau)
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, tau, precision=bddc.BDDC_PREC_FP64)
    assert st[0].n_subdomains == 48
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    flux32, pres32, its32, _, _ = gpu_solve(bddc, [pb], 1e-8, tau, precision=bddc.BDDC_PREC_FP32)
    assert _rel(flux32, ref.flux) <= MIXED_REL and _rel(pres32, ref.pressure) <= MIXED_REL


def test_operator_and_preconditioner_match_oracle(bddc):
    pb = make_config("c1")
    o = BDDCOracle(pb, tau=3.0)
    h = bddc.setup([pb], bddc.default_options(tau=3.0), stream=torch.cuda.current_stream().cuda_stream)
    _, ng, ns = h.sizes()
    assert ng == o.ss.n_gamma and ns == o.ss.N
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(ng)
        p0 = rng.standard_normal(ns)
        q = torch.empty(ng, dtype=torch.float64, device="cuda")
        h.apply_operator(_dev(u), _dev(p0), q)
        qo, _ = o.apply_operator(u, p0)
        assert _rel(q.cpu().numpy(), qo) <= 1e-13
        r = rng.standard_normal(ng)
        z = torch.empty(ng, dtype=torch.float64, device="cuda")
        z0 = torch.empty(ns, dtype=torch.float64, device="cuda")
        h.apply_preconditioner(_dev(r), z, z0)
        zo, z0o = o.precondition(r)
        assert _rel(z.cpu().numpy(), zo) <= 1e-11
        assert _rel(z0.cpu().numpy(), z0o) <= 1e-9
    h.close()


def test_batched_instances_equal_alone(bddc):
    """Instances of different sizes in one persistent launch give bit-identical
    results to their solo solves."""
    pbs = [make_config("c1"), _irregular2d(), make_config("c1", seed=11), make_config("tiny3d")]
    flux, pres, its, st, _ = gpu_solve(bddc, pbs, 1e-8, 4.0)
    fo = np.cumsum([0] + [len(pb.bc_type) for pb in pbs])
    co = np.cumsum([0] + [pb.grid.n_cells for pb in pbs])
    for b, pb in enumerate(pbs):
        fa, pa, ia, _, _ = gpu_solve(bddc, [pb], 1e-8, 4.0)
        assert its[b] == ia[0]
        assert np.array_equal(flux[fo[b]:fo[b + 1]], fa)
        assert np.array_equal(pres[co[b]:co[b + 1]], pa)


@pytest.mark.parametrize("precision", [0, 1])
def test_large_batch_equal_alone_and_oracle(bddc, precision):
    """A batch of 40 channelized 60 x 220 fields (5280 subdomains, more than
    the launch's 4864 warps, so warps hold several subdomains of one
    instance and count their arrivals together, as at the benchmark's batch
    of 256) in one launch: every instance bitwise equal to its solo solve,
    the first and the last against the oracle."""
    B = 40
    pbs = [make_config("c2", seed=2090 + i) for i in range(B)]
    flux, pres, its, st, _ = gpu_solve(bddc, pbs, 1e-8, 10.0, precision=precision)
    assert sum(s.n_subdomains for s in st) == 132 * B
    fo = np.cumsum([0] + [len(pb.bc_type) for pb in pbs])
    co = np.cumsum([0] + [pb.grid.n_cells for pb in pbs])
    for b, pb in enumerate(pbs):
        fa, pa, ia, _, _ = gpu_solve(bddc, [pb], 1e-8, 10.0, precision=precision)
        assert its[b] == ia[0], b
        assert np.array_equal(flux[fo[b]:fo[b + 1]], fa), b
        assert np.array_equal(pres[co[b]:co[b + 1]], pa), b
    bound = MIXED_REL if precision else None
    for b in (0, B - 1):
        ref = BDDCOracle(pbs[b], tau=10.0).solve(tol=1e-8)
        tolb = bound if bound else FP64_REL * max(1.0, ref.kappa)
        assert _rel(flux[fo[b]:fo[b + 1]], ref.flux) <= tolb
        assert _rel(pres[co[b]:co[b + 1]], ref.pressure) <= tolb
        if not precision:
            assert abs(int(its[b]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)


def test_host_and_device_buffers_agree(bddc):
    pb = _irregular2d()
    a = gpu_solve(bddc, [pb], 1e-9, None, device_io=True)
    b = gpu_solve(bddc, [pb], 1e-9, None, device_io=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_subassembled_apply_raw_matches_operator(bddc):
    pb = make_config("tiny3d")
    hs = bddc.HostSetup([pb])
    ng = hs.get("sub_ng")
    n_sub = len(ng)
    slot_off = hs.get("off_slot")
    h = bddc.setup([pb], bddc.default_options(), stream=torch.cuda.current_stream().cuda_stream)
    _, nG, _ = h.sizes()
    u = np.random.default_rng(2).standard_normal(nG)
    q_ref = torch.empty(nG, dtype=torch.float64, device="cuda")
    h.apply_operator(_dev(u), torch.zeros(n_sub, dtype=torch.float64, device="cuda"), q_ref)
    q = torch.full((nG,), np.nan, dtype=torch.float64, device="cuda")
    scratch = torch.empty(int(slot_off[-1]), dtype=torch.float64, device="cuda")
    bddc.subassembled_apply(n_sub, _dev(ng), _dev(slot_off), _dev(hs.get("off_S")), _dev(hs.get("S")),
                            _dev(hs.get("slot_g")), _dev(hs.get("slot_partner")), nG, _dev(u), q, scratch)
    torch.cuda.synchronize()
    assert not torch.isnan(q).any()
    assert torch.allclose(q, q_ref, rtol=1e-13, atol=1e-13 * float(q_ref.abs().max()))
    h.close()


def test_edge_cases(bddc):
    # one subdomain with pressure faces: the interface is the pressure faces
    g = Grid(2, (8, 6, 1), (1.0, 1.0, 1.0))
    t, v = pressure_drop_bc(g)
    rng = np.random.default_rng(3)
    pb = Problem("one", g, 10 ** rng.normal(0, 1, g.n_cells), np.zeros(g.n_cells, np.int32), t, v,
                 np.zeros(g.n_cells))
    ref = BDDCOracle(pb).solve(tol=1e-10)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-10)
    assert _rel(flux, ref.flux) <= 1e-9 and _rel(pres, ref.pressure) <= 1e-9
    # constant k: Steps 1-2 are exact, CG has nothing to do
    g = Grid(2, (12, 12, 1), (1.0, 1.0, 1.0))
    t, v = pressure_drop_bc(g)
    pb = Problem("cf", g, np.full(g.n_cells, 2.0), box_partition(g, (3, 3)), t, v, np.zeros(g.n_cells))
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-10)
    assert its[0] <= 3  # the residual is rounding noise in range(B_0^T)
    nxf = 13 * 12
    assert np.allclose(flux[:nxf], 2.0 / 12.0, rtol=1e-11)
    # iteration limit: status and return code say so, outputs are written
    pb = make_config("c1")
    flux, pres, its, st, rc = gpu_solve(bddc, [pb], 1e-12, None, maxit=3, check=False)
    assert rc == bddc.BDDC_E_NOT_CONVERGED and st[0].status == bddc.BDDC_E_NOT_CONVERGED
    assert its[0] == 3 and np.all(np.isfinite(flux)) and np.all(np.isfinite(pres))
    # invalid input is rejected before any GPU work
    bad = make_config("c1")
    bad.perm = bad.perm.copy()
    bad.perm[0] = np.nan
    with pytest.raises(bddc.BDDCError) as e:
        bddc.setup([bad])
    assert e.value.code == bddc.BDDC_E_PERM


@pytest.mark.parametrize("case", ["c1", "irregular3d_anisotropic", "tiny3d"])
def test_msmfem_and_explicit_constraints_match_oracle(bddc, case):
    """The comparison constraints of Sec. 5 (BDDC_CONSTRAINTS_MSMFEM) and
    caller-given rows (BDDC_CONSTRAINTS_EXPLICIT) on the GPU: FP64 against
    the oracle at tol 1e-8 (iterations, kappa, solution) and 1e-12, the
    mixed path within its bound; the explicit rows also through the serving
    loop, bitwise equal to the solo solve (source-free fields: the library's
    setup distributes the pair sources uniformly)."""
    pb = CASES[case]()
    pb.f = np.zeros(pb.grid.n_cells)
    o = BDDCOracle(pb, constraints="msmfem")
    ref = o.solve(tol=1e-8)
    M = bddc.BDDC_CONSTRAINTS_MSMFEM

    def solve(pbx, tol, prec, mode):
        opt = bddc.default_options(precision=prec, constraints=mode)
        h = bddc.setup([pbx], opt, stream=torch.cuda.current_stream().cuda_stream)
        flux, pres = np.empty(len(pbx.bc_value)), np.empty(pbx.grid.n_cells)
        its = np.zeros(1, dtype=np.int32)
        h.solve(pbx.f, pbx.bc_value, tol, flux, pres, its)
        st = h.stats(0)
        h.close()
        return flux, pres, int(its[0]), st

    flux, pres, its, st = solve(pb, 1e-8, bddc.BDDC_PREC_FP64, M)
    assert st.n_coarse == o.n_coarse
    assert abs(its - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert abs(st.kappa - ref.kappa) <= 0.02 * ref.kappa
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    f32, p32, _, _ = solve(pb, 1e-8, bddc.BDDC_PREC_FP32, M)
    assert _rel(f32, ref.flux) <= MIXED_REL and _rel(p32, ref.pressure) <= MIXED_REL
    ref12 = o.solve(tol=1e-12)
    f12, p12, _, _ = solve(pb, 1e-12, bddc.BDDC_PREC_FP64, M)
    bound = converged_bound(o, ref12)
    assert _rel(f12, ref12.flux) <= bound and _rel(p12, ref12.pressure) <= bound
    # explicit rows: the oracle's MsMFEM rows handed in by the caller
    pb.constraint_rows = [(fa["dofs"], fa["rows"][1]) for fa in o.ss.faces if fa["kind"] == "F"]
    X = bddc.BDDC_CONSTRAINTS_EXPLICIT
    fx, px, itx, stx = solve(pb, 1e-8, bddc.BDDC_PREC_FP64, X)
    assert stx.n_coarse == o.n_coarse
    assert _rel(fx, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    srv = bddc.Server(bddc.default_options(constraints=X), hbm_budget_bytes=4 << 30, max_batch=4)
    t = srv.submit(pb, tol=1e-8)
    srv.wait(t)
    rc, fs, ps, its_s, _, _ = srv.poll(t)
    srv.close()
    assert rc == bddc.BDDC_OK and its_s == itx
    assert np.array_equal(fs, fx) and np.array_equal(ps, px)


@pytest.mark.parametrize("kind,precision", [("batch_dense", 0), ("batch_dense", 1), ("single_sparse", 0)])
def test_autotuned_layout_is_bitwise_equal_and_cached(bddc, kind, precision):
    """bddc_options.autotune: the probe-chosen work layout (the warp ranges'
    weight, the dense coarse unit size) decides which warp or CTA does a
    subdomain's or a coarse row's work, not the order of any sum, so the
    solve is bitwise equal to the heuristic layout's.  The report names one
    of the candidates with its probe times; a second setup with the same
    signature takes the choice from the process cache."""
    if kind == "batch_dense":
        pbs = [make_config("c2", seed=2190 + i) for i in range(6)]
        extra = dict(coarse_solver=bddc.BDDC_COARSE_DENSE)
    else:
        pbs = [_irregular3d()]
        extra = dict(coarse_solver=bddc.BDDC_COARSE_SPARSE)
    stream = torch.cuda.current_stream().cuda_stream
    f = np.concatenate([pb.f for pb in pbs])
    bc = np.concatenate([pb.bc_value for pb in pbs])

    def run(autotune):
        opt = bddc.default_options(tau=4.0, precision=precision, autotune=autotune, **extra)
        h = bddc.setup(pbs, opt, stream=stream)
        flux = torch.empty(len(bc), dtype=torch.float64, device="cuda")
        pres = torch.empty(len(f), dtype=torch.float64, device="cuda")
        its = torch.empty(len(pbs), dtype=torch.int32, device="cuda")
        h.solve(_dev(f), _dev(bc), 1e-10, flux, pres, its)
        torch.cuda.synchronize()
        t = h.tuning()
        rep = (t.tuned, t.from_cache, t.balance_weight, t.coarse_rows, t.probe_ms, t.probe_ms_default)
        out = flux.cpu().numpy(), pres.cpu().numpy(), its.cpu().numpy(), rep
        h.close()
        return out

    heur, tuned, again = run(0), run(1), run(1)
    assert heur[3][:4] == (0, 0, 4096.0, 16)
    assert tuned[3][0] == 1 and tuned[3][1] == 0
    assert tuned[3][2] in (0.0, 1024.0, 4096.0, 16384.0, 65536.0)
    assert tuned[3][3] in ((8, 16, 32) if kind == "batch_dense" else (16,))
    assert 0.0 < tuned[3][4] <= tuned[3][5]
    assert again[3][:2] == (1, 1) and again[3][2:] == tuned[3][2:]
    for out in (tuned, again):
        assert np.array_equal(out[2], heur[2])
        assert np.array_equal(out[0], heur[0])
        assert np.array_equal(out[1], heur[1])


def _split_cases():
    """Subdomains whose S^i exceeds the 32768 entries of one operator-apply
    unit: 8^3-cell boxes (n_Gamma up to 256: three inner faces and a
    pressure face) of a layered 3D field, and seeded boxes of 3-8 cells per
    axis on a 24 x 20 x 16 grid (36 subdomains, 12 of them above the limit,
    n_Gamma up to 287; the c4 partition's shape at a size the oracle takes).
    (2D subdomains that large do not fit the kernel's shared-memory areas.)"""
    from synth.problems import layered_3d
    g3 = Grid(3, (16, 16, 16), (20.0, 10.0, 2.0))
    t3, v3 = pressure_drop_bc(g3)
    p3 = Problem("split3d", g3, layered_3d(g3, 77), box_partition(g3, (2, 2, 2)).astype(np.int32), t3, v3,
                 np.zeros(g3.n_cells))
    gi = Grid(3, (24, 20, 16), (20.0, 10.0, 2.0))
    ti, vi = pressure_drop_bc(gi)
    pi = Problem("split_irr3d", gi, layered_3d(gi, 4085), irregular_box_partition(gi, 4085).astype(np.int32),
                 ti, vi, np.zeros(gi.n_cells))
    return p3, pi


@pytest.mark.parametrize("which", [0, 1])
def test_operator_apply_in_parts_matches_oracle(bddc, which):
    """Subdomains applied as several operator-apply units (their S^i rows in
    output ranges on several warps, the (d, q) partials summed in unit
    order): FP64 and mixed against the oracle, and, in a batch with a small
    instance (the rebalancing kernel), bitwise equal to the solo solve."""
    pb = _split_cases()[which]
    hs = bddc.HostSetup([pb], bddc.default_options(tau=4.0))
    ng = hs.get("sub_ng")
    hs.close()
    assert int((ng.astype(np.int64) ** 2).max()) > 32768
    o = BDDCOracle(pb, tau=4.0)
    ref = o.solve(tol=1e-8)
    flux, pres, its, st, _ = gpu_solve(bddc, [pb], 1e-8, 4.0)
    assert abs(int(its[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(flux, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(pres, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    f32, p32, i32, _, _ = gpu_solve(bddc, [pb], 1e-8, 4.0, precision=bddc.BDDC_PREC_FP32)
    assert _rel(f32, ref.flux) <= MIXED_REL and _rel(p32, ref.pressure) <= MIXED_REL
    for prec, (fa, pa, ia) in ((0, (flux, pres, its)), (1, (f32, p32, i32))):
        pbs = [pb, make_config("c1")]
        fb, pbv, ib, _, _ = gpu_solve(bddc, pbs, 1e-8, 4.0, precision=prec)
        assert ib[0] == ia[0]
        assert np.array_equal(fb[:len(fa)], fa)
        assert np.array_equal(pbv[:len(pa)], pa)

"""GPU parity of the full-space form of the Step-3 operator (BDDC_FORM_FULL).

The persistent kernel with the operator applied as the RT0/P0 mixed
operator on the discrete-harmonic extension of each direction, against the
oracle and against the condensed form on the GPU: the same solution, the
same first CG coefficients and iteration counts, batches equal to single
solves, and the FP64-only restriction.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import make_config  # noqa: E402
from oracle import BDDCOracle  # noqa: E402
from parity import FP64_REL, converged_bound, iteration_slack  # noqa: E402
from test_gpu_parity import _irregular2d, _wells  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bddc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc as b
    return b


def _solve(bddc, pbs, tol, tau, form, coarse=0):
    opt = bddc.default_options(tau=tau, formulation=form, coarse_solver=coarse)
    h = bddc.setup(pbs, opt, stream=torch.cuda.current_stream().cuda_stream)
    f = torch.as_tensor(np.concatenate([pb.f for pb in pbs]), device="cuda")
    bc = torch.as_tensor(np.concatenate([pb.bc_value for pb in pbs]), device="cuda")
    flux = torch.empty(len(bc), dtype=torch.float64, device="cuda")
    pres = torch.empty(len(f), dtype=torch.float64, device="cuda")
    its = torch.empty(len(pbs), dtype=torch.int32, device="cuda")
    h.solve(f, bc, tol, flux, pres, its)
    torch.cuda.synchronize()
    alpha = h.debug_vector("alpha").reshape(len(pbs), -1)
    st = [h.stats(i) for i in range(len(pbs))]
    h.close()
    return flux.cpu().numpy(), pres.cpu().numpy(), its.cpu().numpy(), alpha, st


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = {
    "c1": lambda: make_config("c1"),
    "irregular2d": _irregular2d,
    "c2": lambda: make_config("c2", seed=2091),
    "tiny3d": lambda: make_config("tiny3d"),
    "c1_wells": lambda: _wells(make_config("c1")),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_full_form_matches_oracle_and_condensed(bddc, case):
    pb = CASES[case]()
    tau = 10.0
    o = BDDCOracle(pb, tau=tau)
    ref = o.solve(tol=1e-8)
    f2, p2, it2, al2, st2 = _solve(bddc, [pb], 1e-8, tau, bddc.BDDC_FORM_FULL)
    f1, p1, it1, al1, _ = _solve(bddc, [pb], 1e-8, tau, bddc.BDDC_FORM_CONDENSED)
    assert st2[0].status == 0
    assert abs(int(it2[0]) - ref.iterations) <= iteration_slack(ref.iterations, ref.kappa)
    assert abs(int(it2[0]) - int(it1[0])) <= iteration_slack(ref.iterations, ref.kappa)
    assert _rel(f2, ref.flux) <= FP64_REL * max(1.0, ref.kappa)
    assert _rel(p2, ref.pressure) <= FP64_REL * max(1.0, ref.kappa)
    # the same operator up to rounding: the CG coefficients agree before the
    # two finite-precision runs drift apart
    n = min(5, int(it1[0]), int(it2[0]))
    assert np.allclose(al2[0, :n], al1[0, :n], rtol=1e-9, atol=0)
    assert st2[0].true_relres <= 1e-7
    # converged: within the converged bound of the oracle
    ref = o.solve(tol=1e-12)
    f2, p2, _, _, _ = _solve(bddc, [pb], 1e-12, tau, bddc.BDDC_FORM_FULL)
    bound = converged_bound(o, ref)
    assert _rel(f2, ref.flux) <= bound
    assert _rel(p2, ref.pressure) <= bound


def test_full_form_batch_equals_single_solves(bddc):
    pbs = [make_config("c1"), _irregular2d(), make_config("c2", seed=2093)]
    fb, pbp, itb, _, _ = _solve(bddc, pbs, 1e-8, 10.0, bddc.BDDC_FORM_FULL)
    fo = po = 0
    for i, pb in enumerate(pbs):
        f1, p1, it1, _, _ = _solve(bddc, [pb], 1e-8, 10.0, bddc.BDDC_FORM_FULL)
        assert itb[i] == it1[0]
        assert np.array_equal(fb[fo:fo + len(f1)], f1)
        assert np.array_equal(pbp[po:po + len(p1)], p1)
        fo += len(f1)
        po += len(p1)


def test_full_form_with_the_sparse_coarse_solver(bddc):
    pb = make_config("tiny3d")
    f2, p2, it2, _, _ = _solve(bddc, [pb], 1e-10, 10.0, bddc.BDDC_FORM_FULL, coarse=bddc.BDDC_COARSE_SPARSE)
    f1, p1, it1, _, _ = _solve(bddc, [pb], 1e-10, 10.0, bddc.BDDC_FORM_CONDENSED, coarse=bddc.BDDC_COARSE_SPARSE)
    assert abs(int(it2[0]) - int(it1[0])) <= 1
    assert _rel(f2, f1) <= 1e-8 and _rel(p2, p1) <= 1e-8


def test_full_form_needs_fp64_on_the_device(bddc):
    pb = make_config("c1")
    opt = bddc.default_options(formulation=bddc.BDDC_FORM_FULL, precision=bddc.BDDC_PREC_FP32)
    with pytest.raises(bddc.BDDCError) as e:
        bddc.setup([pb], opt, stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.code == bddc.BDDC_E_INVALID_ARG

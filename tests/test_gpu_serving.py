"""Serving loop (continuous batching) on the GPU: results are bitwise those
of the same problem solved alone, memory admission holds the HBM budget,
a bad request fails alone, and requests submitted while a batch runs join
later batches."""

import os
import sys
import time

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from synth import make_config  # noqa: E402
from synth.problems import serving_request  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bddc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1901_02090_gb300 import bddc as b
    return b


def _alone(bddc, pb, opt, tol):
    h = bddc.setup([pb], opt)
    flux = np.empty(len(pb.bc_type))
    pres = np.empty(pb.grid.n_cells)
    its = np.zeros(1, dtype=np.int32)
    rc = h.solve(pb.f, pb.bc_value, tol, flux, pres, its, check=False)
    st = h.stats(0)
    h.close()
    return rc, flux, pres, int(its[0]), st


def _collect(srv, tickets, timeout=300.0):
    out = {}
    t_end = time.time() + timeout
    for t in tickets:
        assert srv.wait(t, max(1.0, t_end - time.time())), "request did not finish"
        out[t] = srv.poll(t)
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_alone(bddc, precision):
    """Requests of different sizes (30-60 x 110-220 cells, random pressure
    direction) solved in shared batches give bitwise the results of the same
    problem set up and solved alone."""
    opt = bddc.default_options(tau=10.0, precision=precision)
    srv = bddc.Server(opt, hbm_budget_bytes=8 << 30, max_batch=8)
    pbs = [serving_request(i) for i in range(10)]
    tickets = [srv.submit(pb, tol=1e-8) for pb in pbs]
    res = _collect(srv, tickets)
    info = srv.info()
    srv.close()
    assert info.completed == 10 and info.failed == 0
    sizes = set()
    for pb, t in zip(pbs, tickets):
        rc, flux, pres, its, st, rinfo = res[t]
        assert rc == bddc.BDDC_OK
        sizes.add(rinfo.batch_size)
        rc1, flux1, pres1, its1, st1 = _alone(bddc, pb, opt, 1e-8)
        assert rc1 == bddc.BDDC_OK
        assert its == its1 == st.iterations
        assert np.array_equal(flux, flux1) and np.array_equal(pres, pres1)
        assert st.kappa == pytest.approx(st1.kappa, rel=1e-12)
        assert 0 <= rinfo.queue_ms <= rinfo.latency_ms and rinfo.solve_ms > 0
    assert max(sizes) > 1  # requests shared launches


def test_served_result_matches_oracle(bddc):
    from oracle import BDDCOracle
    pb = serving_request(3)
    ref = BDDCOracle(pb, tau=10.0).solve(tol=1e-8)
    srv = bddc.Server(bddc.default_options(tau=10.0, precision=0), max_batch=4)
    t = srv.submit(pb, tol=1e-8)
    rc, flux, pres, its, st, _ = _collect(srv, [t])[t]
    srv.close()
    assert rc == bddc.BDDC_OK
    rel = np.linalg.norm(flux - ref.flux) / np.linalg.norm(ref.flux)
    assert rel <= 1e-8 * max(1.0, ref.kappa)


def test_budget_admission_and_splitting(bddc):
    """A budget that holds about one 60 x 220 request at a time: every request
    still completes, in several batches, and the device memory of the
    admitted batches never exceeds the budget."""
    opt = bddc.default_options(tau=10.0, precision=1)
    pb = make_config("c2", seed=2090)
    # footprint of one request, measured through a one-request server
    srv = bddc.Server(opt, hbm_budget_bytes=8 << 30, max_batch=1)
    t = srv.submit(pb)
    _collect(srv, [t])
    one = srv.info().device_bytes_peak
    srv.close()
    budget = int(1.5 * one)
    srv = bddc.Server(opt, hbm_budget_bytes=budget, max_batch=8)
    pbs = [make_config("c2", seed=2090 + i) for i in range(5)]
    tickets = [srv.submit(p) for p in pbs]
    res = _collect(srv, tickets)
    info = srv.info()
    srv.close()
    assert all(res[t][0] == bddc.BDDC_OK for t in tickets)
    assert info.batches >= 3 and info.device_bytes_peak <= budget
    assert info.device_bytes_in_use == 0


def test_bad_request_fails_alone(bddc):
    opt = bddc.default_options(tau=10.0, precision=1)
    good = serving_request(1)
    bad = serving_request(2)
    bad.perm = bad.perm.copy()
    bad.perm[5] = -1.0  # not a permeability
    srv = bddc.Server(opt, max_batch=8)
    tg = srv.submit(good)
    tb = srv.submit(bad)
    res = _collect(srv, [tg, tb])
    srv.close()
    assert res[tb][0] == bddc.BDDC_E_PERM
    assert res[tg][0] == bddc.BDDC_OK
    rc1, flux1, _, _, _ = _alone(bddc, good, opt, 1e-8)
    assert np.array_equal(res[tg][1], flux1)


def test_requests_arriving_during_a_solve_join_later_batches(bddc):
    """Continuous batching: requests submitted while earlier ones are on the
    GPU are admitted into later launches, and all come back."""
    opt = bddc.default_options(tau=10.0, precision=1)
    srv = bddc.Server(opt, max_batch=16)
    first = [srv.submit(serving_request(100 + i)) for i in range(4)]
    time.sleep(0.05)
    later = []
    for i in range(12):
        later.append(srv.submit(serving_request(200 + i)))
        time.sleep(0.01)
    res = _collect(srv, first + later)
    info = srv.info()
    # a collected ticket is released
    assert bddc.lib.bddc_poll(srv._h, first[0], None, None, None, None, None) == bddc.BDDC_E_INVALID_ARG
    srv.close()
    assert all(r[0] == bddc.BDDC_OK for r in res.values())
    ids = {res[t][5].batch_id for t in first + later}
    assert info.batches == len(ids) >= 2
    assert info.completed == 16

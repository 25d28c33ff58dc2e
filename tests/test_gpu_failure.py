"""Failure detection on the GPU without a fault: the solve kernel's grid
barriers wait with a time limit; a wait that runs out sets an error flag
that ends the kernel, the host reports BDDC_E_TIMEOUT, and the device
context stays usable.  The wait is made to run out with a barrier that one
CTA never enters (bddc_debug_barrier_timeout), not by faulting or hanging
anything."""

import time

import numpy as np
import pytest

from synth import make_config


def test_barrier_timeout_rejects_invalid_arguments():
    from paper_1901_02090_gb300 import bddc
    for limit, n in [(0, 2), (-1, 2), (61_000_000_000, 2), (50_000_000, 1), (50_000_000, 2000)]:
        assert bddc.lib.bddc_debug_barrier_timeout(limit, n) == bddc.BDDC_E_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("n_ctas", [2, 64])
def test_barrier_wait_runs_out_and_context_stays_usable(n_ctas):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    t0 = time.time()
    rc = bddc.lib.bddc_debug_barrier_timeout(50_000_000, n_ctas)  # 50 ms limit
    dt = time.time() - t0
    assert rc == bddc.BDDC_E_TIMEOUT
    assert dt < 5.0
    # the context still works: a regular solve afterwards
    pb = make_config("c1")
    h = bddc.setup([pb], bddc.default_options(tau=4.0), stream=torch.cuda.current_stream().cuda_stream)
    flux, pres = np.empty(len(pb.bc_value)), np.empty(pb.grid.n_cells)
    assert h.solve(pb.f, pb.bc_value, 1e-10, flux, pres) == bddc.BDDC_OK
    assert h.stats(0).true_relres < 1e-8
    h.close()

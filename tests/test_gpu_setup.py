"""The dense local maps computed on the GPU (the path bddc_setup and the
serving loop take) against the host computation of the same algorithm:
S^i, G_pre, G_post and everything built from them (F, Psi, the coarse
inverse, the adaptive constraints) agree to rounding."""

import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from synth import make_config  # noqa: E402
from test_gpu_parity import CASES  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bddc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1901_02090_gb300 import bddc as b
    return b


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("case", ["c1", "tiny3d", "irregular2d", "irregular3d_anisotropic", "c2"])
@pytest.mark.parametrize("tau", [0.0, 10.0])
def test_device_local_maps_match_host(bddc, case, tau):
    pb = make_config("c2", seed=2093) if case == "c2" else CASES[case]()
    opt = bddc.default_options(tau=tau, precision=0)
    host = bddc.HostSetup([pb], opt)
    dev = bddc.HostSetup([pb], opt, device=True)
    # the structure does not depend on where the maps were computed
    for name in ("sub_ng", "sub_m", "off_S", "off_Gpost", "slot_g", "cslot_c"):
        assert np.array_equal(host.get(name), dev.get(name)), name
    for name in ("S", "Gpre", "Gpost"):
        assert _rel(dev.get(name), host.get(name)) <= 1e-11, name
    for name in ("F", "P", "P64", "Kinv"):
        assert _rel(dev.get(name), host.get(name)) <= 1e-9, name
    assert dev.get("inst_omega")[0] == pytest.approx(host.get("inst_omega")[0], rel=1e-8)

"""GPU test of bddc_subassembled_apply_noalloc, the allocation-free entry
point for callers that cannot call cudaMalloc (its scratch is a fixed array
in the library's device memory).

It must give the same result as bddc_subassembled_apply with caller-owned
scratch, on two calls in a row (the shared array keeps the previous call's
contents, which the next call must not depend on).  The file is named so that
pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import make_config  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_noalloc_apply_matches_scratch_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    pbs = [make_config("c1"), make_config("tiny3d")]
    hs = bddc.HostSetup(pbs)
    ng = hs.get("sub_ng")
    n_sub = len(ng)
    slot_off = hs.get("off_slot")
    n_slots = int(slot_off[-1])
    assert n_slots <= bddc.NOALLOC_MAX_SLOTS
    n_gamma = int(hs.get("inst_ng").sum())
    args = (n_sub, _dev(ng), _dev(slot_off), _dev(hs.get("off_S")), _dev(hs.get("S")),
            _dev(hs.get("slot_g")), _dev(hs.get("slot_partner")), n_gamma)
    rng = np.random.default_rng(7)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        u = _dev(rng.standard_normal(n_gamma) * (10.0 ** call))
        ref = torch.full((n_gamma,), np.nan, dtype=torch.float64, device="cuda")
        scratch = torch.empty(n_slots, dtype=torch.float64, device="cuda")
        bddc.subassembled_apply(*args, u, ref, scratch, stream=stream)
        out = torch.full((n_gamma,), np.nan, dtype=torch.float64, device="cuda")
        bddc.subassembled_apply_noalloc(*args, u, out, stream=stream)
        torch.cuda.synchronize()
        assert not torch.isnan(out).any()
        assert torch.allclose(out, ref, rtol=1e-13, atol=1e-13 * float(ref.abs().max()))


def test_noalloc_apply_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    big = bddc.NOALLOC_MAX_SLOTS + 1
    ng = _dev(np.array([1], dtype=np.int32))
    slot_off = _dev(np.array([0, big], dtype=np.int64))
    dummy_i = _dev(np.zeros(1, dtype=np.int32))
    dummy_l = _dev(np.zeros(1, dtype=np.int64))
    dummy_d = _dev(np.zeros(1))
    with pytest.raises(bddc.BDDCError) as e:
        bddc.subassembled_apply_noalloc(1, ng, slot_off, dummy_l, dummy_d, dummy_i, dummy_i, 1, dummy_d,
                                        torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert e.value.code == bddc.BDDC_E_INVALID_ARG
    assert "exceed" in str(e.value)

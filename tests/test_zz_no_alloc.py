"""GPU test of bddc_subassembled_apply_noalloc, the allocation-free entry
point for callers that cannot call cudaMalloc (code inside a memory pool or
arena that owns the device memory, or a loop that may not allocate after
start-up); its scratch is a fixed array in the library's device memory.

It must give the same result as bddc_subassembled_apply with caller-owned
scratch, on two calls in a row: the first on a two-instance layout, the
second on a smaller one-instance layout, so the second call runs over a
shared array that still holds the first call's (larger) contents.  Offsets
that are not the prefix sums of the local sizes are rejected on the host,
before any kernel runs.  The file is named so that pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import make_config  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _layout(bddc, pbs):
    hs = bddc.HostSetup(pbs)
    ng = hs.get("sub_ng")
    slot_off = hs.get("off_slot")
    n_gamma = int(hs.get("inst_ng").sum())
    args = (len(ng), _dev(ng), _dev(slot_off), _dev(hs.get("off_S")), _dev(hs.get("S")),
            _dev(hs.get("slot_g")), _dev(hs.get("slot_partner")), n_gamma)
    return args, int(slot_off[-1]), n_gamma


def test_noalloc_apply_matches_scratch_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    rng = np.random.default_rng(7)
    stream = torch.cuda.current_stream().cuda_stream
    layouts = [[make_config("c1"), make_config("tiny3d")], [make_config("tiny3d", seed=5)]]
    sizes = []
    for call, pbs in enumerate(layouts):
        args, n_slots, n_gamma = _layout(bddc, pbs)
        assert n_slots <= bddc.NOALLOC_MAX_SLOTS
        sizes.append(n_slots)
        u = _dev(rng.standard_normal(n_gamma) * (10.0 ** call))
        ref = torch.full((n_gamma,), np.nan, dtype=torch.float64, device="cuda")
        scratch = torch.empty(n_slots, dtype=torch.float64, device="cuda")
        bddc.subassembled_apply(*args, u, ref, scratch, stream=stream)
        out = torch.full((n_gamma,), np.nan, dtype=torch.float64, device="cuda")
        bddc.subassembled_apply_noalloc(*args, u, out, stream=stream)
        torch.cuda.synchronize()
        assert not torch.isnan(out).any()
        assert torch.allclose(out, ref, rtol=1e-13, atol=1e-13 * float(ref.abs().max()))
    assert sizes[1] < sizes[0]


def test_noalloc_apply_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    big = bddc.NOALLOC_MAX_SLOTS + 1
    # one subdomain of 1024 dofs per entry of ng would need more subdomains;
    # a consistent layout past the limit: ng all 1024
    n_sub = big // 1024 + 1
    ng = np.full(n_sub, 1024, dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(ng)]).astype(np.int64)
    assert off[-1] > bddc.NOALLOC_MAX_SLOTS
    dummy_i = _dev(np.zeros(1, dtype=np.int32))
    dummy_l = _dev(np.zeros(n_sub, dtype=np.int64))
    dummy_d = _dev(np.zeros(1))
    with pytest.raises(bddc.BDDCError) as e:
        bddc.subassembled_apply_noalloc(n_sub, _dev(ng), _dev(off), dummy_l, dummy_d, dummy_i, dummy_i, 1, dummy_d,
                                        torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert e.value.code == bddc.BDDC_E_INVALID_ARG
    assert "exceed" in str(e.value)


@pytest.mark.parametrize("bad", ["non_monotone", "size_mismatch", "nonzero_start", "ng_too_large"])
def test_noalloc_apply_rejects_inconsistent_offsets(bad):
    """Offsets that are not the prefix sums of ng (which would let one
    subdomain's slots run past another's, or past the fixed array) are
    rejected on the host before any kernel runs; so are local sizes outside
    0..1024.  Both entry points apply the same check."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_02090_gb300 import bddc
    args, n_slots, n_gamma = _layout(bddc, [make_config("c1")])
    n_sub, ng_d, off_d = args[0], args[1], args[2]
    ng = ng_d.cpu().numpy().copy()
    off = off_d.cpu().numpy().copy()
    if bad == "non_monotone":
        off[2], off[3] = off[3], off[2]
    elif bad == "size_mismatch":
        off[1] += 1
    elif bad == "nonzero_start":
        off = off + 4
    else:
        ng[0] = 2048
    bad_args = (n_sub, _dev(ng), _dev(off)) + args[3:]
    u = _dev(np.ones(n_gamma))
    for call in ("noalloc", "scratch"):
        out = torch.full((n_gamma,), np.nan, dtype=torch.float64, device="cuda")
        with pytest.raises(bddc.BDDCError) as e:
            if call == "noalloc":
                bddc.subassembled_apply_noalloc(*bad_args, u, out)
            else:
                scratch = torch.empty(n_slots + 64, dtype=torch.float64, device="cuda")
                bddc.subassembled_apply(*bad_args, u, out, scratch)
        assert e.value.code == bddc.BDDC_E_INVALID_ARG
        torch.cuda.synchronize()
        assert torch.isnan(out).all()  # nothing was launched

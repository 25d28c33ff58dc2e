"""The full-space form of the Step-3 operator (BDDC_FORM_FULL), on the host.

The setup exports, per interface slot, the cell of its subdomain on the
slot's face, the face's RT0 mass coefficient in that cell and the cell's
other face along the same axis.  With the interface columns of G_post (the
discrete-harmonic extension) they give the mixed operator of Sec. 2 applied
to the extended direction.  Pinned to the oracle's discretization (which
cell, which faces, the entries of the RT0 mass block) and to the condensed
form S^i d + d_s sigma p_0 on random directions; the PCG that uses it
reaches the oracle's solution.
"""

import numpy as np
import pytest

from oracle import BDDCOracle
from oracle.discretization import Discretization
from packed_emulation import Packed, emulate_solve, full_form_apply
from paper_1901_02090_gb300 import bddc
from synth import make_config
from test_native_setup import CASES


def _setup(pb, **kw):
    kw.setdefault("formulation", bddc.BDDC_FORM_FULL)
    return Packed(bddc.HostSetup([pb], bddc.default_options(tau=4.0, **kw)))


@pytest.mark.parametrize("case", sorted(CASES))
def test_face_data_match_the_oracle_discretization(case):
    pb = CASES[case]()
    P = _setup(pb)
    disc = Discretization(pb)
    cf, fc = disc.cell_faces, disc.face_cells()
    for s in range(P.n_sub):
        sl = P.slots(s)
        ng, ni, nc = int(P.sub_ng[s]), int(P.sub_ni[s]), int(P.sub_nc[s])
        faces = np.concatenate([P.g_fid[P.slot_g[sl]], P.int_fid[P.off_int[s]:P.off_int[s] + ni]])
        cells = P.cell_gid[P.off_cell[s]:P.off_cell[s] + nc]
        for k in range(ng):
            e = int(faces[k])
            a = int(disc.face_axis(e))
            code = int(P.slot_fcell[sl[k]])
            K = int(cells[abs(code) - 1])
            below, above = fc[e]
            # +: the face is the lower face of K (K lies above it)
            assert (K == above) if code > 0 else (K == below)
            assert cf[K, a, 0 if code > 0 else 1] == e
            opp = int(cf[K, a, 1 if code > 0 else 0])
            o = int(P.slot_fopp[sl[k]])
            if o >= 0:
                assert faces[o] == opp
            else:
                assert opp not in set(faces.tolist()) and pb.bc_type[opp] == 0
            M = disc.cell_mass_block(K, a)
            assert abs(P.slot_fk[sl[k]] / 3.0 - M[0, 0]) <= 1e-14 * M[0, 0]


@pytest.mark.parametrize("case", sorted(CASES) + ["c2"])
def test_full_form_equals_the_condensed_operator(case):
    pb = make_config("c2", seed=2090) if case == "c2" else CASES[case]()
    P = _setup(pb)
    rng = np.random.default_rng(1)
    for s in range(P.n_sub):
        sl = P.slots(s)
        ng = int(P.sub_ng[s])
        S = P.mat(P.S, P.off_S, s, ng, ng)
        for _ in range(2):
            d, dp = rng.standard_normal(ng), rng.standard_normal()
            q1 = S @ d + P.slot_dsig[sl] * dp
            q2 = full_form_apply(P, s, d, dp)
            assert np.abs(q1 - q2).max() <= 1e-12 * np.abs(q1).max()


@pytest.mark.parametrize("case", ["c1", "irregular2d", "tiny3d"])
def test_full_form_pcg_reaches_the_oracle_solution(case):
    pb = CASES[case]()
    P = _setup(pb)
    o = BDDCOracle(pb, tau=4.0)
    r = o.solve(tol=1e-12)
    flux, pres, its, al, _ = emulate_solve(P, pb.f, pb.bc_value, 1e-12, full_form=True)
    assert np.linalg.norm(flux - r.flux) <= 1e-9 * np.linalg.norm(r.flux)
    assert np.linalg.norm(pres - r.pressure) <= 1e-8 * np.linalg.norm(r.pressure)
    # the same iterates as the condensed form: the first CG coefficients agree
    # (the setup of the full form carries everything the condensed form uses)
    _, _, its1, al1, _ = emulate_solve(P, pb.f, pb.bc_value, 1e-12)
    n = min(6, len(al[0]), len(al1[0]))
    assert np.allclose(al[0][:n], al1[0][:n], rtol=1e-9, atol=0)


def test_full_form_needs_fp64():
    pb = CASES["c1"]()
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([pb], bddc.default_options(formulation=bddc.BDDC_FORM_FULL, precision=bddc.BDDC_PREC_FP32))
    assert e.value.code == bddc.BDDC_E_INVALID_ARG
    with pytest.raises(bddc.BDDCError) as e:
        bddc.HostSetup([pb], bddc.default_options(formulation=7))
    assert e.value.code == bddc.BDDC_E_INVALID_ARG


def test_condensed_setup_builds_no_face_data():
    P = Packed(bddc.HostSetup([CASES["c1"]()], bddc.default_options(tau=4.0)))
    assert len(P.slot_fk) == 0 and len(P.slot_fopp) == 0 and len(P.slot_fcell) == 0

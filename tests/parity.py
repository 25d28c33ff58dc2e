"""Tolerances shared by the parity tests (GPU or emulation vs the oracle)."""

import math

# FP64 path: relative flux and pressure error against the oracle at the same
# tolerance (spec bound), and at tol 1e-12 where both are converged
# (converged_bound).
FP64_REL = 1e-8
CONVERGED_REL = 1e-10
# mixed path (FP32 subdomain correction and coarse basis): bound after the
# FP64 CG has converged to 1e-8
MIXED_REL = 1e-6


def iteration_slack(iterations, kappa):
    """Allowed difference in CG iterations: one, or 5% of the count when the
    preconditioned operator has kappa > 50.  Two FP64 CG runs whose
    operators differ only by rounding follow the same path for about ten
    steps and then drift apart; where the residual curve is flat near the
    tolerance the crossing moves by a few steps (the oracle run with and
    without the pressure rescaling D, mathematically identical, differs the
    same way; the MsMFEM-constrained c1 field, kappa 94, ends 2 of 48 steps
    apart on the GPU).  The adaptive runs (kappa < 30) keep one step."""
    if kappa <= 50:
        return 1
    return max(1, int(math.floor(0.05 * iterations)))


def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def converged_bound(oracle, ref):
    """Bound on the relative flux and pressure difference of two FP64 solves
    at tol 1e-12 (GPU against the oracle result ``ref``): CONVERGED_REL plus
    twice the oracle's own distance from the direct solve of the assembled
    saddle system.  Each converged solution is within its rounding error of
    the exact one; on the 1e7-contrast channelized fields the oracle itself
    stays ~2e-10 from the direct solve, so a fixed 1e-10 would measure the
    conditioning, not the parity.  On mildly heterogeneous cases the bound is
    about 1e-10."""
    from oracle import direct_solve
    fd, pd = direct_solve(oracle.disc)
    e = max(_rel(ref.flux, fd), _rel(ref.pressure, pd))
    return CONVERGED_REL + 2.0 * e

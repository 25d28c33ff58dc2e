"""CPU FP64 oracle for adaptive BDDC on mixed RT0/P0 Darcy flow.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method of Sousedik, "On adaptive BDDC for the flow in
heterogeneous porous media" (arXiv:1901.02090).  Only the test-suite, the
smoke check and the benchmark's CPU-baseline leg may import it.  The GPU
library never calls, links or reads anything here, and nothing here imports
the GPU library: the two share only the seeded input generators of ``synth``.

Modules
-------
discretization  RT0 fluxes and P0 pressures on a Cartesian grid (Sec. 2):
                bilinear forms a and b, the right-hand side, boundary data,
                the global saddle-point system (Sec. 4, eq. (system)) and its
                direct solution.
substructure    subdomains, interface, faces, restriction maps, the scaling
                operator E and the initial flux constraints (Sec. 3,
                Assumption 1, Sec. 4.1 eq. (C^i)).
bddc            local constrained saddle-point solves, the coarse basis and
                coarse problem, Algorithm 1 (three steps), Algorithm 2 (BDDC
                preconditioner), PCG with the Lanczos condition estimate, and
                the pressure block rescaling D (Sec. 4).
adaptive        the local generalized eigenproblems on pairs of adjacent
                subdomains (Sec. 3.1 eqs. (eigenvalue-problem-local-matrix)),
                Algorithm 3 and the indicator omega-tilde (eq. (indicator)).
msmfem          the multiscale (MsMFEM-style) constraints of the comparison
                in Sec. 5 (pair Darcy problems with sources +-w) and
                caller-given constraint rows.

Parity status of each function is stated in its docstring; every function
here is pinned by the CPU tests in ``tests/test_oracle_*.py`` except where a
docstring says "parity unpinned".
"""

from .discretization import Discretization, direct_solve  # noqa: F401
from .substructure import Substructuring  # noqa: F401
from .bddc import BDDCOracle, SolveResult, lanczos_condition  # noqa: F401
from .adaptive import adaptive_constraints  # noqa: F401

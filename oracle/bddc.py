"""Two-level BDDC for the mixed problem, Algorithms 1 and 2 (oracle).

Test infrastructure only (see the package docstring).

Everything here follows the paper's definitions with dense or sparse direct
solves of the local saddle-point problems; nothing is blocked, fused or
reordered beyond those definitions.

Local problems of subdomain i (local flux dofs ordered interface first, then
interior; cells; multipliers).  With the rescaled divergence block d_i B^i
(Sec. 4, eq. (system-scaled)) and the pressure constraint row C_Q^i (cell
volumes, Sec. 4.1):

  Stokes-harmonic operator (Sec. 3, definition of P and (I - P)W):
      K_S = [[A, dB^T, 0], [dB, 0, C_Q^T], [0, C_Q, 0]]
  constrained local operator (Sec. 4.1, eq. (C^i)):
      K_C = [[A, dB^T, C_U^T, 0], [dB, 0, 0, C_Q^T], [C_U, 0, 0, 0],
             [0, C_Q, 0, 0]]

S^i is the Schur complement of K_S onto the interface fluxes (the energy of
the Stokes-harmonic extension, Sec. 3.1 "S^{ij}").  The coarse basis Psi^i is
the flux part of K_C^{-1} applied to unit vectors in the C_U rows
(Algorithm 2 step 1 via the standard BDDC coarse basis); the subdomain
correction of Algorithm 2 step 2 is the flux part of K_C^{-1} applied to the
weighted residual.
"""

from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import Discretization
from .substructure import Substructuring


class BreakdownError(RuntimeError):
    pass


@dataclasses.dataclass
class SolveResult:
    flux: np.ndarray          # all global faces
    pressure: np.ndarray      # per cell
    iterations: int
    kappa: float              # Lanczos estimate (Sec. 5)
    relres: list              # relative residual history
    alphas: list
    betas: list
    u0_gamma: np.ndarray      # Step 1 interface values
    u_star: np.ndarray        # after Step 2, all global faces
    u0: np.ndarray            # Step 1 coarse component, all global faces


def lanczos_condition(alphas, betas):
    """Condition number estimate from the CG coefficients (Sec. 5: "computed
    from the Lanczos sequence in conjugate gradients").  Reading (the formula
    is not printed): the standard CG-Lanczos tridiagonal
    T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1},
    T_{k,k+1} = sqrt(beta_k)/alpha_k, and kappa = lambda_max / lambda_min."""
    m = len(alphas)
    if m == 0:
        return 1.0
    T = np.zeros((m, m))
    for k in range(m):
        T[k, k] = 1.0 / alphas[k] + (betas[k - 1] / alphas[k - 1] if k > 0 else 0.0)
        if k + 1 < m:
            T[k, k + 1] = T[k + 1, k] = np.sqrt(betas[k]) / alphas[k]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


class _Local:
    """Factorised local operators of one subdomain."""

    def __init__(self, sub, C_U, cell_volume):
        nf, nc = len(sub.faces), len(sub.cells)
        ng = sub.n_gamma
        m = C_U.shape[0]
        self.nf, self.nc, self.ng, self.m = nf, nc, ng, m
        dB = sub.d * sub.B
        vol = np.full((nc, 1), cell_volume)  # C_Q: row of cell volumes (Sec. 3)
        A = sub.A
        # Stokes-harmonic operator K_S
        KS = np.block([
            [A, dB.T, np.zeros((nf, 1))],
            [dB, np.zeros((nc, nc)), vol],
            [np.zeros((1, nf)), vol.T, np.zeros((1, 1))],
        ])
        self.KS = KS
        rest = np.arange(ng, KS.shape[0])
        gam = np.arange(ng)
        Krr = sp.csc_matrix(KS[np.ix_(rest, rest)])
        self.lu_rest = spla.splu(Krr)
        Krg = KS[np.ix_(rest, gam)]
        X = self.lu_rest.solve(Krg) if ng > 0 else np.zeros((len(rest), 0))
        # S^i: Schur complement of K_S onto the interface fluxes
        S = KS[np.ix_(gam, gam)] - KS[np.ix_(gam, rest)] @ X
        self.S = 0.5 * (S + S.T)
        # Stokes-harmonic extension of interface values: interior fluxes and
        # the mean-free pressure it carries
        self.H = np.vstack([np.eye(ng), -X[: nf - ng]])      # nf x ng
        self.P = -X[nf - ng: nf - ng + nc]                     # nc x ng
        # constrained operator K_C
        CU = np.zeros((m, nf))
        CU[:, :ng] = C_U
        KC = np.block([
            [A, dB.T, CU.T, np.zeros((nf, 1))],
            [dB, np.zeros((nc, nc)), np.zeros((nc, m)), vol],
            [CU, np.zeros((m, nc)), np.zeros((m, m)), np.zeros((m, 1))],
            [np.zeros((1, nf)), vol.T, np.zeros((1, m)), np.zeros((1, 1))],
        ])
        self.lu_C = spla.splu(sp.csc_matrix(KC))
        # coarse basis: unit coarse value in each C_U row
        rhs = np.zeros((KC.shape[0], m))
        rhs[nf + nc: nf + nc + m, :] = np.eye(m)
        sol = self.lu_C.solve(rhs) if m > 0 else rhs
        self.Psi = sol[:nf, :]                                  # nf x m
        # interior problem of Step 2 (interior fluxes, cells, multiplier)
        ni = nf - ng
        AII = A[ng:, ng:]
        dBI = dB[:, ng:]
        KI = np.block([
            [AII, dBI.T, np.zeros((ni, 1))],
            [dBI, np.zeros((nc, nc)), vol],
            [np.zeros((1, ni)), vol.T, np.zeros((1, 1))],
        ])
        self.lu_I = spla.splu(sp.csc_matrix(KI))
        self.A, self.dB = A, dB

    def delta_solve(self, r_gamma):
        """Algorithm 2 step 2: the Stokes-harmonic local flux with zero flux
        coarse dofs responding to the functional r on the interface."""
        rhs = np.zeros(self.nf + self.nc + self.m + 1)
        rhs[: self.ng] = r_gamma
        return self.lu_C.solve(rhs)[: self.nf]


class BDDCOracle:
    """Adaptive BDDC solver for the RT0/P0 Darcy system (oracle).

    Parameters
    ----------
    problem : synth.Problem
    tau : float or None
        Adaptive threshold of Algorithm 3; None or inf for the initial
        (face-average) constraints only.
    scaling : "multiplicity" (default, Sec. 5) or "stiffness".
    pressure_scaling : apply the block rescaling D of Sec. 4.
    constraints : None (the initial net-flux constraints, plus Algorithm 3
        when tau is given), "msmfem" (plus one MsMFEM row per face, the
        comparison method of Sec. 5; tau is ignored) or "explicit" (plus the
        rows of ``explicit_rows``: a list of (global face ids, coefficients),
        each on one face).
    """

    def __init__(self, problem, tau=None, scaling="multiplicity", pressure_scaling=True, constraints=None,
                 explicit_rows=None):
        self.problem = problem
        self.disc = Discretization(problem)
        self.ss = Substructuring(self.disc, problem.partition, scaling=scaling,
                                 pressure_scaling=pressure_scaling)
        self.tau = tau
        self.omega_tilde = None
        self.face_eigenvalues = None
        if constraints in ("msmfem", "explicit"):
            from .msmfem import explicit_constraints, msmfem_constraints
            rows = msmfem_constraints(self) if constraints == "msmfem" else \
                explicit_constraints(self, explicit_rows or [])
            for fidx, new_rows in sorted(rows.items()):
                self.ss.add_face_rows(fidx, new_rows)
            self.n_added = sum(len(r) for r in rows.values())
            self._build(initial=False)
            return
        if constraints is not None:
            raise ValueError(f"unknown constraints {constraints!r}")
        self._build(initial=True)
        if tau is not None and np.isfinite(tau):
            from .adaptive import adaptive_constraints
            rows, omega, eigs = adaptive_constraints(self, tau)
            for fidx, new_rows in rows.items():
                self.ss.add_face_rows(fidx, new_rows)
            self.omega_tilde, self.face_eigenvalues = omega, eigs
            self._build(initial=False)

    # ---- setup -------------------------------------------------------------
    def _build(self, initial):
        ss = self.ss
        cons = ss.local_constraints()
        self.local = [_Local(sub, C, self.disc.vol) for sub, (C, _) in zip(ss.subs, cons)]
        self.cids = [ids for _, ids in cons]
        self._coarse_problem()

    def _coarse_problem(self):
        """Coarse saddle-point matrix over (W_Pi, Q_0), Algorithm 1 step 1 and
        Algorithm 2 step 1: a(psi_j, psi_l) summed over subdomains, and
        b(psi_j, 1_i) for the subdomain constants.  Pure-flux problems add the
        zero-mean condition of Q_0 by a bordering multiplier."""
        ss = self.ss
        nc = ss.n_coarse_flux
        N = ss.N
        Kc = np.zeros((nc, nc))
        Bc = np.zeros((N, nc))
        for sub, loc, ids in zip(ss.subs, self.local, self.cids):
            Psi = loc.Psi
            Kc[np.ix_(ids, ids)] += Psi.T @ loc.A @ Psi
            Bc[sub.id, ids] += np.ones(loc.nc) @ loc.dB @ Psi
        self.pure_flux = not np.any(self.disc.dirichlet)
        if self.pure_flux:
            v = np.array([sub.d * len(sub.cells) * self.disc.vol for sub in ss.subs])
            K = np.block([
                [Kc, Bc.T, np.zeros((nc, 1))],
                [Bc, np.zeros((N, N)), v[:, None]],
                [np.zeros((1, nc)), v[None, :], np.zeros((1, 1))],
            ])
        else:
            K = np.block([[Kc, Bc.T], [Bc, np.zeros((N, N))]])
        self.Kc_full = K
        self.coarse_lu = sla.lu_factor(K)
        self.n_coarse = nc + N

    def coarse_solve(self, rhs_flux, rhs_pressure):
        ss = self.ss
        nc, N = ss.n_coarse_flux, ss.N
        rhs = np.zeros(self.Kc_full.shape[0])
        rhs[:nc] = rhs_flux
        rhs[nc: nc + N] = rhs_pressure
        sol = sla.lu_solve(self.coarse_lu, rhs)
        return sol[:nc], sol[nc: nc + N]

    # ---- interface operators ------------------------------------------------
    def restrict(self, v):
        return [v[self.ss.gpos[sub.gamma]] for sub in self.ss.subs]

    def assemble(self, parts, weighted=False):
        out = np.zeros(self.ss.n_gamma)
        for sub, p in zip(self.ss.subs, parts):
            np.add.at(out, self.ss.gpos[sub.gamma], sub.weights * p if weighted else p)
        return out

    def apply_operator(self, u, p0):
        """The reduced operator of eqs. (corr-reduced-1)-(corr-reduced-2):
        flux part S u + B_0^T p_0 (S = sum_i R_i^T S^i R_i), and B_0 u."""
        ss = self.ss
        q = np.zeros(ss.n_gamma)
        bu = np.zeros(ss.N)
        for sub, loc, ul in zip(ss.subs, self.local, self.restrict(u)):
            contrib = loc.S @ ul + sub.d * sub.sigma * p0[sub.id]
            np.add.at(q, ss.gpos[sub.gamma], contrib)
            bu[sub.id] = sub.d * sub.sigma @ ul
        return q, bu

    def precondition(self, r):
        """Algorithm 2 (BDDC preconditioner): (r_B, 0) -> (w_hat, p_0)."""
        ss = self.ss
        rl = [sub.weights * x for sub, x in zip(ss.subs, self.restrict(r))]
        # step 1: coarse correction, rhs <r_B, E z_Pi>
        rc = np.zeros(ss.n_coarse_flux)
        for loc, ids, x in zip(self.local, self.cids, rl):
            np.add.at(rc, ids, loc.Psi[: loc.ng].T @ x)
        wc, p0 = self.coarse_solve(rc, np.zeros(ss.N))
        # step 2: subdomain corrections; step 3: sum and average
        parts = []
        for loc, ids, x in zip(self.local, self.cids, rl):
            w_pi = loc.Psi @ wc[ids]
            w_delta = loc.delta_solve(x)
            parts.append((w_pi + w_delta)[: loc.ng])
        return self.assemble(parts, weighted=True), p0

    # ---- Algorithm 1 ---------------------------------------------------------
    def solve(self, tol=1e-8, maxit=1000, residual_norm="l2"):
        ss, disc = self.ss, self.disc
        g_all = disc.face_rhs()
        g_gamma = g_all[ss.gamma]
        cell_rhs = disc.cell_rhs()

        # Step 1: coarse component (eqs. (two-level-nested_coarse-1/2))
        rc = np.zeros(ss.n_coarse_flux)
        rp = np.zeros(ss.N)
        for sub, loc, ids, gl in zip(ss.subs, self.local, self.cids, self.restrict(g_gamma)):
            np.add.at(rc, ids, loc.Psi[: loc.ng].T @ (sub.weights * gl))
            rp[sub.id] = sub.d * np.sum(cell_rhs[sub.cells])
        wc, _ = self.coarse_solve(rc, rp)
        u0_gamma = self.assemble([loc.Psi[: loc.ng] @ wc[ids] for loc, ids in zip(self.local, self.cids)],
                                 weighted=True)

        # Step 2: subdomain components
        u_star_loc, p2_loc = [], []
        for sub, loc, ug in zip(ss.subs, self.local, self.restrict(u0_gamma)):
            u0_full = loc.H @ ug                      # u_0 = E w_0 is Stokes harmonic
            ng, ni = loc.ng, loc.nf - loc.ng
            rhs = np.concatenate([
                -(loc.A @ u0_full)[ng:],
                sub.d * cell_rhs[sub.cells] - loc.dB @ u0_full,
                [0.0],
            ])
            sol = loc.lu_I.solve(rhs)
            u_star = u0_full.copy()
            u_star[ng:] += sol[:ni]
            u_star_loc.append(u_star)
            p2_loc.append(sol[ni: ni + loc.nc])

        # Step 3: reduced right-hand side <f*, v> = <g, v> - a(u*, v), v in W_hat
        fstar = g_gamma.copy()
        for sub, loc, us in zip(ss.subs, self.local, u_star_loc):
            np.add.at(fstar, ss.gpos[sub.gamma], -(loc.H.T @ (loc.A @ us)))

        # absolute floor: f* is a difference of two terms of size `scale`;
        # below 1e-14 * scale it is rounding noise and CG has nothing to do
        scale = np.linalg.norm(g_gamma) + np.linalg.norm(g_gamma - fstar)
        x, xp, it, relres, alphas, betas = self.pcg(fstar, tol, maxit, residual_norm,
                                                    floor=1e-14 * scale)

        # post-correction: interiors and pressures
        flux = np.zeros(disc.n_faces)
        pressure = np.zeros(disc.n_cells)
        u_star_glob = np.zeros(disc.n_faces)
        u0_glob = np.zeros(disc.n_faces)
        for sub, loc, us, p2, xl, u0l in zip(ss.subs, self.local, u_star_loc, p2_loc,
                                             self.restrict(x), self.restrict(u0_gamma)):
            u = us + loc.H @ xl
            flux[sub.faces] = u
            u_star_glob[sub.faces] = us
            u0_glob[sub.faces] = loc.H @ u0l
            pbar = xp[sub.id] + p2 + loc.P @ xl
            pressure[sub.cells] = sub.d * pbar
        kappa = lanczos_condition(alphas, betas)
        return SolveResult(flux, pressure, it, kappa, relres, alphas, betas,
                           u0_gamma, u_star_glob, u0_glob)

    def pcg(self, b, tol, maxit, residual_norm="l2", floor=0.0):
        """CG on the pairs (w_hat, p_0) of eqs. (corr-reduced-1/2) with the BDDC
        preconditioner; x_0 = 0 is balanced and the preconditioner's output is
        balanced, so CG is valid (Sec. 3).  Stops when the relative residual
        falls below tol (Sec. 5).  Reading: the Euclidean norm of the
        flux-residual of the reduced system (its pressure part is zero), or
        the preconditioned norm sqrt(r.z) if residual_norm == "precond".

        The flux iterates do not depend on the pressure components (the
        preconditioner maps B_0^T q to (0, q)), and the pressure iterate only
        converges together with the flux.  Reading for the end of the
        iteration: once the flux has converged (stopping test, the rounding
        floor, or (r, z) vanishing relative to its first value) the pressure
        takes one last coarse correction x_p += z_p from the final residual,
        so the returned pressure solves the reduced system for the returned
        flux."""
        ss = self.ss
        x = np.zeros(ss.n_gamma)
        xp = np.zeros(ss.N)
        r = b.copy()
        z, zp = self.precondition(r)
        rho = float(r @ z)
        rho0 = rho
        nrm = (lambda r, rho: np.sqrt(max(rho, 0.0))) if residual_norm == "precond" else \
              (lambda r, rho: np.linalg.norm(r))
        r0 = nrm(r, rho)
        relres, alphas, betas = [1.0], [], []
        it = 0
        # M is positive semi-definite, so (r, z) <= 0 at the start is a
        # rounded zero: r lies in range(B_0^T) and only the pressure is left
        if np.linalg.norm(r) > floor and rho > 0.0:
            d, dp = z.copy(), zp.copy()
            for k in range(maxit):
                q, _ = self.apply_operator(d, dp)
                dq = float(d @ q)
                if not dq > 0:
                    raise BreakdownError("(d, Kd) <= 0")
                alpha = rho / dq
                x += alpha * d
                xp += alpha * dp
                r -= alpha * q
                alphas.append(alpha)
                it = k + 1
                z, zp = self.precondition(r)
                rho_new = float(r @ z)
                res = nrm(r, rho_new) / r0
                relres.append(res)
                if res <= tol or np.linalg.norm(r) <= floor or rho_new <= RHO_FLUX_CONVERGED * rho0:
                    break
                if not rho_new > 0:
                    raise BreakdownError("(r, z) <= 0")
                beta = rho_new / rho
                betas.append(beta)
                rho = rho_new
                d = z + beta * d
                dp = zp + beta * dp
        # final pressure correction from the last residual
        xp += zp
        return x, xp, it, relres, alphas, betas


# (r, z) below this fraction of its first value means the flux part of the
# residual is rounding noise (the remaining residual is B_0^T of a pressure)
RHO_FLUX_CONVERGED = 1e-24

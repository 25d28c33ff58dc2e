"""Adaptive selection of flux constraints (Sec. 3.1, Algorithm 3), oracle.

Test infrastructure only (see the package docstring).

For every pair of adjacent subdomains i, j (sharing a face Gamma^{ij}):

* the pair space is Gamma^i x Gamma^j (Stokes-harmonic functions are
  represented by their interface values) with the energy
  S^{ij} = diag(S^i, S^j);
* E^{ij} averages the two copies of the dofs of Gamma^{ij} with the weights
  of E and leaves every other dof unchanged, so (I - E^{ij}) is nonzero only on
  the rows and columns of Gamma^{ij};
* the constraint matrix is C = C_U^{ij} (I - E^{ij}), where C_U^{ij} holds the
  initial constraint rows of the face Gamma^{ij} only (reading of eq.
  (def-Wtilde-dual): "the initial constraints at the face Gamma^{ij}");
* eq. (eigenvalue-problem-local-matrix),
  Pi (I-E)^T S (I-E) Pi w = lambda Pi S Pi w, is solved in the range of the
  orthogonal projection Pi onto null C: with Z an orthonormal basis of null C
  (from an SVD of C), Z^T (I-E)^T S (I-E) Z y = lambda Z^T S Z y, by a dense
  symmetric-definite eigensolver;
* Algorithm 3: with lambda sorted decreasingly, the k eigenvectors with
  lambda > tau give the rows c_l = w_l^T Pi (I-E)^T S (I-E) Pi of
  eq. (constraints); each splits as [c^i, -c^i] and the half c^i (over the
  face dofs, global orientation) is added to both C_U^i and C_U^j;
* reading of the unstated row normalisation: the new rows are
  orthonormalised (modified Gram-Schmidt) against the face's existing rows,
  which changes the basis of the constraints, not the space W-tilde;
* omega^{ij} is the largest eigenvalue left (lambda_{k+1}, or 0), and
  omega-tilde (eq. (indicator)) is the maximum over all pairs (reported as
  computed, not clipped at 1).
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pair_problem(oracle, face):
    """Matrices of the local eigenproblem of one face: returns
    (S_ij, I_minus_E, C, face_positions_i, face_positions_j)."""
    ss = oracle.ss
    i, j = face["i"], face["j"]
    si, sj = ss.subs[i], ss.subs[j]
    li, lj = oracle.local[i], oracle.local[j]
    ni, nj = si.n_gamma, sj.n_gamma
    n = ni + nj
    S = np.zeros((n, n))
    S[:ni, :ni] = li.S
    S[ni:, ni:] = lj.S
    loc_i = {int(e): k for k, e in enumerate(si.gamma)}
    loc_j = {int(e): k for k, e in enumerate(sj.gamma)}
    pi = np.array([loc_i[int(e)] for e in face["dofs"]])
    pj = np.array([loc_j[int(e)] for e in face["dofs"]]) + ni
    IE = np.zeros((n, n))
    wi = si.weights[pi]
    wj = sj.weights[pj - ni]
    # (I - E)w on i's copy: w^i - (w_i w^i + w_j w^j) = w_j (w^i - w^j)
    IE[pi, pi] = wj
    IE[pi, pj] = -wj
    IE[pj, pj] = wi
    IE[pj, pi] = -wi
    # initial constraint rows of the face on both copies (A8 reading)
    CU = np.zeros((2, n))
    CU[0, pi] = face["rows"][0]
    CU[1, pj] = face["rows"][0]
    C = CU @ IE
    return S, IE, C, pi, pj


def null_basis(C, rtol=1e-12):
    """Orthonormal basis of null C from an SVD."""
    n = C.shape[1]
    if C.size == 0:
        return np.eye(n)
    U, s, Vt = np.linalg.svd(C)
    rank = int(np.sum(s > rtol * (s[0] if s.size else 1.0)))
    return Vt[rank:].T


def face_eigen(oracle, face):
    """Eigenvalues (descending) and eigenvectors w_l of
    eq. (eigenvalue-problem-local-matrix) for one face, plus the pair
    matrices."""
    S, IE, C, pi, pj = pair_problem(oracle, face)
    Z = null_basis(C)
    Pi = Z @ Z.T
    Aop = IE.T @ S @ IE
    lhs = Z.T @ Aop @ Z
    rhs = Z.T @ S @ Z
    lam, Y = sla.eigh(0.5 * (lhs + lhs.T), 0.5 * (rhs + rhs.T))
    order = np.argsort(lam)[::-1]
    lam, Y = lam[order], Y[:, order]
    W = Z @ Y
    return lam, W, dict(S=S, IE=IE, Pi=Pi, Aop=Aop, pi=pi, pj=pj)


def _orthonormalize(existing, new_rows, drop_tol=1e-10):
    basis = [r / np.linalg.norm(r) for r in existing]
    out = []
    for r in new_rows:
        v = r.astype(np.float64).copy()
        n0 = np.linalg.norm(v)
        for b in basis:
            v -= (b @ v) * b
        for b in basis:            # second pass for stability
            v -= (b @ v) * b
        nv = np.linalg.norm(v)
        if n0 > 0 and nv > drop_tol * n0:
            v /= nv
            basis.append(v)
            out.append(v)
    return out


def adaptive_constraints(oracle, tau):
    """Algorithm 3 on every face between two subdomains.

    Returns (rows, omega_tilde, eigenvalues): rows maps a face index to the
    list of new rows (over that face's dofs), eigenvalues maps a face index
    to its descending eigenvalues.
    """
    ss = oracle.ss
    rows, eigs = {}, {}
    omega = 0.0
    for fidx, face in enumerate(ss.faces):
        if face["kind"] != "F":
            continue
        lam, W, mats = face_eigen(oracle, face)
        eigs[fidx] = lam
        k = int(np.sum(lam > tau)) if np.isfinite(tau) else 0
        omega_ij = float(lam[k]) if k < len(lam) else 0.0
        omega = max(omega, omega_ij)
        if k == 0:
            continue
        new = []
        for ell in range(k):
            w = W[:, ell]
            c = (mats["Pi"] @ w) @ mats["Aop"] @ mats["Pi"]
            new.append(c[mats["pi"]])       # the half c^i on the face dofs
        new = _orthonormalize(face["rows"], new)
        if new:
            rows[fidx] = new
    return rows, omega, eigs

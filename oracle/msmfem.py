"""Constraints inspired by the multiscale mixed finite element method (MsMFEM),
the comparison method of Sec. 5 (oracle).

Test infrastructure only (see the package docstring).

For every face Gamma^{ij} between two subdomains the paper solves a local
Darcy problem on the pair of subdomains -- the local counterpart of the
problem of Sec. 2 -- with the source w_i on Omega^i, -w_j on Omega^j and no
flow through the boundary of the pair, and adds the flux values the
solution takes on the face dofs as one more constraint of that face, beside
the initial net-flux constraint.  The source distribution is w_i = 1/|Omega^i|
except in a subdomain with sources (a well), where it is f / int_{Omega^i} f.

Readings (the passage is terse):
* M1: the no-flow condition holds on the whole boundary of Omega^i u Omega^j
  (the printed "boundary of Omega^i n Omega^j" would be the face itself,
  through which the flow has to pass); every face of the pair's cells that
  is not between two cells of the pair carries zero flux, including faces
  on the boundary of the domain.
* M2: the pair problem determines the pressure up to a constant; it is
  fixed by a zero mean (a cell-volume row, as for the local problems of
  Sec. 3).
* M3: "a subdomain containing a well" is one with a nonzero integral of f;
  there w = f / int f.  (A subdomain whose sources integrate to zero gets
  the uniform distribution.)
* M4: the new row is orthonormalised against the face's existing rows, as
  the adaptive rows are (reading A9 of the adaptive constraints).
* Rows given by the caller (the EXPLICIT constraint mode of the library) go
  through the same orthonormalisation; each must lie on the dofs of one face.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .adaptive import _orthonormalize


def pair_source(disc, cells, sign):
    """Source density w on the cells of one subdomain (Sec. 5): 1/|Omega^i|
    uniformly, or f / int f where the subdomain's sources integrate to a
    nonzero value (reading M3); multiplied by sign (+1 for Omega^i, -1 for
    Omega^j)."""
    f = disc.f[cells]
    total = float(np.sum(f) * disc.vol)
    if total != 0.0:
        w = f / total
    else:
        w = np.full(len(cells), 1.0 / (len(cells) * disc.vol))
    return sign * w


def pair_flux(oracle, face):
    """The local Darcy problem of one face on Omega^i u Omega^j (Sec. 5;
    readings M1, M2): returns the flux on the face dofs (global orientation,
    in the order of face["dofs"]) and the full local solution
    (faces, flux, cells, pressure)."""
    ss, disc = oracle.ss, oracle.disc
    i, j = face["i"], face["j"]
    cells = np.concatenate([ss.subs[i].cells, ss.subs[j].cells])
    in_pair = np.zeros(disc.n_cells, dtype=bool)
    in_pair[cells] = True
    fc = ss.face_cells
    # faces with both cells in the pair (all others carry no flux, M1)
    cand = np.unique(disc.cell_faces[cells].reshape(-1))
    both = (fc[cand, 0] >= 0) & (fc[cand, 1] >= 0)
    cand = cand[both]
    faces = cand[in_pair[fc[cand, 0]] & in_pair[fc[cand, 1]]]
    A, B = disc.assemble(cells, faces)
    w = np.concatenate([pair_source(disc, ss.subs[i].cells, 1.0), pair_source(disc, ss.subs[j].cells, -1.0)])
    nf, nc = len(faces), len(cells)
    vol = np.full((nc, 1), disc.vol)
    K = np.block([
        [A, B.T, np.zeros((nf, 1))],
        [B, np.zeros((nc, nc)), vol],
        [np.zeros((1, nf)), vol.T, np.zeros((1, 1))],
    ])
    rhs = np.zeros(nf + nc + 1)
    rhs[nf: nf + nc] = -w * disc.vol  # <w, q_c> = -int_c w (Sec. 2, eq. (rhs))
    sol = sla.solve(K, rhs)
    u, p = sol[:nf], sol[nf: nf + nc]
    pos = {int(e): n for n, e in enumerate(faces)}
    row = np.array([u[pos[int(e)]] for e in face["dofs"]])
    return row, (faces, u, cells, p)


def msmfem_constraints(oracle):
    """One MsMFEM row per face between two subdomains (Sec. 5): the pair
    problem's flux on the face dofs, orthonormalised against the face's
    existing rows (M4).  Returns {face index: [row]}."""
    rows = {}
    for fidx, face in enumerate(oracle.ss.faces):
        if face["kind"] != "F":
            continue
        row, _ = pair_flux(oracle, face)
        new = _orthonormalize(face["rows"], [row])
        if new:
            rows[fidx] = new
    return rows


def explicit_constraints(oracle, explicit):
    """Caller rows: ``explicit`` is a list of (global face ids, coefficients);
    each row lies on the dofs of one face Gamma^{ij} and is orthonormalised
    against that face's rows (M4).  Returns {face index: [rows]}."""
    ss = oracle.ss
    where = {}
    for fidx, fa in enumerate(ss.faces):
        if fa["kind"] == "F":
            for n, e in enumerate(fa["dofs"]):
                where[int(e)] = (fidx, n)
    grouped = {}
    for faces, coef in explicit:
        loc = [where.get(int(e)) for e in faces]
        if any(x is None for x in loc) or len({x[0] for x in loc}) != 1:
            raise ValueError("an explicit constraint row must lie on the dofs of one face between two subdomains")
        fidx = loc[0][0]
        row = np.zeros(len(ss.faces[fidx]["dofs"]))
        for (fi, n), c in zip(loc, coef):
            row[n] += c
        grouped.setdefault(fidx, []).append(row)
    rows = {}
    for fidx, new in grouped.items():
        kept = _orthonormalize(ss.faces[fidx]["rows"], new)
        if kept:
            rows[fidx] = kept
    return rows

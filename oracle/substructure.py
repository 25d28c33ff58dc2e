"""Substructuring data for BDDC (oracle).  Test infrastructure only.

Sec. 3: non-overlapping subdomains Omega^i; Gamma^i are the flux degrees of
freedom of Omega^i shared with another subdomain; a face Gamma^{ij} is the
intersection Gamma^i n Gamma^j.  With RT0 there are faces only (no corners or
edges).  W^i is the space of local fluxes; U_I the interior fluxes; local
vectors keep the global orientation of each flux (so continuity across the
interface is equality of the two copies).

Initial constraints (Assumption 1, eq. (starting_flux_constraint)): one
zero-net-flux row per face.  Its coefficient on a face dof is the sign of
that dof's +axis normal with respect to the outward normal of the lower-id
subdomain, so the row value is the net flux out of that subdomain through the
face and both sides use the same row in global orientation.

Pressure faces (reading; the paper assumes Gamma_N empty): every face with a
prescribed pressure is treated as an interface dof with a single owner
(multiplicity 1), and each group of such faces of one subdomain on one side
of the box gets its own net-flux coarse dof.  Then U_I still has no flux
through the subdomain boundary, b(u_I, q_0) = 0 keeps holding, the coarse
pressure space is all subdomain constants, and the operator (I - E) vanishes
on those faces.

Scaling E (Sec. 3, Remark "scaling"): a weighted average of the copies of an
interface dof; multiplicity weights are 1/2 on shared faces and 1 on pressure
faces.  Stiffness weights (an option, Sec. 5) are the face-wise share of
the local diagonals, sum_F A^i_ee / sum_F (A^i_ee + A^j_ee), constant along
each face Gamma^{ij} (the Remark "scaling" of Sec. 3).
"""

from __future__ import annotations

import numpy as np

from .discretization import Discretization


class Subdomain:
    """Local data of one subdomain."""

    def __init__(self, sid, cells, faces, n_interface):
        self.id = sid
        self.cells = cells              # global cell ids
        self.faces = faces              # local flux dofs: interface first, then interior
        self.n_gamma = n_interface      # interface dofs are faces[:n_gamma]
        self.gamma = faces[:n_interface]
        self.interior = faces[n_interface:]
        self.A = None                   # local (unassembled) a-form matrix
        self.B = None                   # local b-form matrix (cells x faces)
        self.d = 1.0                    # pressure block scaling (Sec. 4)
        self.weights = None             # E weights on interface dofs
        self.sigma = None               # (B^i)^T 1 on interface dofs
        self.coarse_rows = []           # list of (global coarse id, row over gamma)


class Substructuring:
    """Subdomains, interface numbering, faces and initial coarse dofs."""

    def __init__(self, disc: Discretization, partition, scaling="multiplicity",
                 pressure_scaling=True, matrices=True):
        self.disc = disc
        part = np.asarray(partition, dtype=np.int64)
        if part.shape != (disc.n_cells,):
            raise ValueError("partition must have one entry per cell")
        ids = np.unique(part)
        if ids[0] != 0 or ids[-1] != len(ids) - 1:
            raise ValueError("subdomain ids must be 0..N-1 with none empty")
        self.part = part
        self.N = len(ids)
        fc = disc.face_cells()
        self.face_cells = fc
        owner = np.where(fc >= 0, part[np.maximum(fc, 0)], -1)  # (n_faces, 2)
        self.face_owner = owner
        free = disc.free
        shared = free & (owner[:, 0] >= 0) & (owner[:, 1] >= 0) & (owner[:, 0] != owner[:, 1])
        dir_faces = disc.dirichlet
        self.is_interface = shared | dir_faces
        self.gamma = np.nonzero(self.is_interface)[0]          # global interface dofs
        self.n_gamma = len(self.gamma)
        self.gpos = -np.ones(disc.n_faces, dtype=np.int64)
        self.gpos[self.gamma] = np.arange(self.n_gamma)

        self.subs = []
        for s in range(self.N):
            cells = np.nonzero(part == s)[0]
            faces = np.unique(disc.cell_faces[cells].reshape(-1))
            faces = faces[free[faces]]
            itf = faces[self.is_interface[faces]]
            inn = faces[~self.is_interface[faces]]
            sub = Subdomain(s, cells, np.concatenate([itf, inn]), len(itf))
            self._check_connected(sub)
            self.subs.append(sub)
        self._build_faces()
        if not matrices:
            return
        for sub in self.subs:
            sub.A, sub.B = disc.assemble(sub.cells, sub.faces)

        # pressure block rescaling D (Sec. 4, eq. (system-scaled)); reading:
        # mean of the diagonal of the local, unassembled A^i
        for sub in self.subs:
            sub.d = float(np.mean(np.diag(sub.A))) if pressure_scaling else 1.0

        # sigma_i = (B^i)^T 1 on interface dofs: -1 if the dof's +normal
        # points out of subdomain i, +1 if into it
        for sub in self.subs:
            sub.sigma = (np.ones(len(sub.cells)) @ sub.B)[: sub.n_gamma]

        self._build_weights(scaling)

    def _check_connected(self, sub):
        """A subdomain must be face-connected (its local problem must fix the
        pressure up to one constant)."""
        n = len(sub.cells)
        if n == 0:
            raise ValueError("empty subdomain")
        pos = {int(c): r for r, c in enumerate(sub.cells)}
        fc = self.disc.face_cells()
        adj = [[] for _ in range(n)]
        for e in sub.interior:
            a, b = fc[e]
            adj[pos[int(a)]].append(pos[int(b)])
            adj[pos[int(b)]].append(pos[int(a)])
        seen = np.zeros(n, bool)
        stack = [0]
        seen[0] = True
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if not seen[w]:
                    seen[w] = True
                    stack.append(w)
        if not seen.all():
            raise ValueError(f"subdomain {sub.id} is not connected")

    def _build_faces(self):
        """Faces Gamma^{ij} and pressure-face groups, with their net-flux rows."""
        owner = self.face_owner
        disc = self.disc
        faces = {}
        for e in self.gamma:
            o0, o1 = owner[e]
            if disc.dirichlet[e]:
                s = o0 if o0 >= 0 else o1
                ax = int(disc.face_axis(e))
                side = 1 if owner[e, 1] < 0 else 0
                faces.setdefault(("D", s, ax, side), []).append(e)
            else:
                i, j = min(o0, o1), max(o0, o1)
                faces.setdefault(("F", i, j), []).append(e)
        self.faces = []          # list of dicts
        for key in sorted(faces, key=lambda k: (k[0] != "F",) + tuple(k[1:])):
            dofs = np.array(sorted(faces[key]), dtype=np.int64)
            if key[0] == "F":
                i, j = key[1], key[2]
                # +1 where the dof's +normal points out of subdomain i
                coef = np.where(owner[dofs, 0] == i, 1.0, -1.0)
                self.faces.append(dict(kind="F", i=i, j=j, dofs=dofs, coef=coef))
            else:
                s = key[1]
                coef = np.where(owner[dofs, 0] == s, 1.0, -1.0)
                self.faces.append(dict(kind="D", i=s, j=-1, dofs=dofs, coef=coef))
        self.n_faces_shared = sum(1 for f in self.faces if f["kind"] == "F")
        # initial coarse flux dofs: one per face / pressure-face group
        for sub in self.subs:
            sub.coarse_rows = []
        for cid, fa in enumerate(self.faces):
            fa["coarse_ids"] = [cid]
            fa["rows"] = [fa["coef"].copy()]
        self.n_coarse_flux = len(self.faces)

    def _build_weights(self, scaling):
        """Weights of E on each subdomain's interface dofs.

        Multiplicity: 1/2 on a face shared by two subdomains, 1 on pressure
        faces.  Stiffness (Sec. 5, the jumps experiment): the share of the
        diagonal of the local a-form matrices, taken per face Gamma^{ij}
        rather than per dof -- w_i = sum_{e in Gamma^{ij}} A^i_ee /
        sum_{e in Gamma^{ij}} (A^i_ee + A^j_ee) on every dof of the face.
        Reading: the Remark "scaling" of Sec. 3 states that the initial
        net-flux constraints do not allow the weights of E to vary along an
        interface if u* is to satisfy b(u*, q) = <f, q>; with weights that
        vary along a face Step 2 leaves u* non-conservative and Step 3
        cannot repair it.  Where the permeability jumps are aligned with the
        subdomains (the case the paper uses stiffness scaling for) the
        diagonal is constant along each face and the two definitions
        coincide; for RT0 they are then the rho-scaling k_i^-1 / (k_i^-1 +
        k_j^-1) (Sec. 5)."""
        if scaling not in ("multiplicity", "stiffness"):
            raise ValueError(f"unknown scaling {scaling!r}")
        for sub in self.subs:
            sub.weights = np.ones(sub.n_gamma)
        for fa in self.faces:
            if fa["kind"] != "F":
                continue  # pressure faces: a single owner, weight 1
            si, sj = self.subs[fa["i"]], self.subs[fa["j"]]
            loc_i = {int(e): n for n, e in enumerate(si.gamma)}
            loc_j = {int(e): n for n, e in enumerate(sj.gamma)}
            pi = np.array([loc_i[int(e)] for e in fa["dofs"]])
            pj = np.array([loc_j[int(e)] for e in fa["dofs"]])
            if scaling == "multiplicity":
                wi = wj = 0.5
            else:
                ai = float(np.sum(np.diag(si.A)[pi]))
                aj = float(np.sum(np.diag(sj.A)[pj]))
                wi, wj = ai / (ai + aj), aj / (ai + aj)
            si.weights[pi] = wi
            sj.weights[pj] = wj

    # ---- coarse dof rows per subdomain ------------------------------------
    def local_constraints(self):
        """For each subdomain the matrix C_U^i (rows over its interface dofs)
        and the global coarse ids of its rows (Sec. 4.1, eq. (C^i))."""
        out = []
        for sub in self.subs:
            loc = {int(e): n for n, e in enumerate(sub.gamma)}
            rows, ids = [], []
            for fa in self.faces:
                if fa["i"] != sub.id and fa["j"] != sub.id:
                    continue
                for cid, row in zip(fa["coarse_ids"], fa["rows"]):
                    r = np.zeros(sub.n_gamma)
                    for e, v in zip(fa["dofs"], row):
                        r[loc[int(e)]] = v
                    rows.append(r)
                    ids.append(cid)
            out.append((np.array(rows).reshape(len(rows), sub.n_gamma), np.array(ids, dtype=np.int64)))
        return out

    def add_face_rows(self, face_index, new_rows):
        """Append adaptive rows (over the face's dofs) to one face; they get
        new global coarse ids."""
        fa = self.faces[face_index]
        for r in new_rows:
            fa["rows"].append(np.asarray(r, dtype=np.float64))
            fa["coarse_ids"].append(self.n_coarse_flux)
            self.n_coarse_flux += 1

    def counts(self):
        """Table 1 quantities: N, n_Gamma (shared dofs), n_f, n_c (initial)."""
        n_shared = int(np.sum(self.is_interface & ~self.disc.dirichlet))
        return dict(N=self.N, n_gamma=n_shared, n_f=self.n_faces_shared,
                    n_c=self.n_faces_shared + self.N)

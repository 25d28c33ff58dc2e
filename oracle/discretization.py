"""RT0 x P0 mixed discretisation of Darcy flow on a Cartesian grid (oracle).

Test infrastructure only (see the package docstring).

Model (Sec. 2, eqs. (problem-1)-(problem-4)): k^{-1} u + grad p = 0,
div u = f, p = p_N on Gamma_N, u.n = g_E on Gamma_E.

Discrete forms (Sec. 2, eqs. (a), (b), (rhs)):
    a(u, v) = int k^{-1} u . v,   b(u, q) = -int (div u) q,
    <f, q>  = -int f q.
One flux degree of freedom per face: the total normal flux through it,
positive along +axis.  One pressure per cell (indicator basis).

On an h_x x h_y (x h_z) box the velocity of the flux basis function of the
lower a-face is (1 - xi_a) / |face| e_a and of the upper a-face xi_a / |face|
e_a, xi_a in [0, 1] the local coordinate.  Exact integration gives the cell
mass block k_a^{-1} (h_a^2 / |cell|) [[1/3, 1/6], [1/6, 1/3]] on the two
a-faces, with no coupling between axes (k diagonal).  The divergence of the
cell is (flux through upper face) - (flux through lower face), hence
B[cell, upper] = -1, B[cell, lower] = +1.

Boundary data.  Faces with a prescribed flux are removed from the unknowns
(only g_E = 0, as assumed in Sec. 2).  A prescribed pressure p_N on a face
contributes -p_N (v . n) to the flux equation of that face: +p_N on a face
at the minimum side of an axis, -p_N at the maximum side (reading of the
paper, which itself assumes Gamma_N empty; the BDDC treatment of such faces
is described in ``substructure``).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synth.problems import Grid, Problem, face_axis_counts

MASS_DIAG = 1.0 / 3.0
MASS_OFF = 1.0 / 6.0


class Discretization:
    """Face/cell numbering, local cell matrices and the global system."""

    def __init__(self, problem: Problem):
        self.problem = problem
        g: Grid = problem.grid
        self.grid = g
        self.dim = g.dim
        self.nx, self.ny, self.nz = g.n
        self.n_cells = g.n_cells
        counts = face_axis_counts(g)
        self.face_offset = np.concatenate([[0], np.cumsum(counts)])
        self.n_faces = int(self.face_offset[-1])
        self.vol = g.cell_volume
        perm = np.asarray(problem.perm, dtype=np.float64)
        if perm.ndim == 1:
            perm = np.repeat(perm[:, None], self.dim, axis=1)
        if perm.shape != (self.n_cells, self.dim):
            raise ValueError("perm must have shape (n_cells,) or (n_cells, dim)")
        if not np.all(np.isfinite(perm)) or np.any(perm <= 0):
            raise ValueError("permeability must be finite and positive")
        self.perm = perm
        self.bc_type = np.asarray(problem.bc_type, dtype=np.int8)
        self.bc_value = np.asarray(problem.bc_value, dtype=np.float64)
        if np.any((self.bc_type == 0) & (self.bc_value != 0.0)):
            raise ValueError("only zero prescribed flux (no flow) is supported")
        self.f = np.asarray(problem.f, dtype=np.float64)
        self._cell_faces = self._build_cell_faces()
        # free faces: inside the domain or with a prescribed pressure
        self.free = self.bc_type != 0
        self.dirichlet = self.bc_type == 1

    # ---- numbering -------------------------------------------------------
    def cell_ijk(self, c):
        c = np.asarray(c)
        return c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)

    def face_id(self, axis, i, j, k):
        ext = [self.nx, self.ny, self.nz]
        ext[axis] += 1
        return self.face_offset[axis] + i + ext[0] * (j + ext[1] * k)

    def _build_cell_faces(self):
        """(n_cells, dim, 2) global face ids: [c, a, 0] lower, [c, a, 1] upper."""
        c = np.arange(self.n_cells)
        i, j, k = self.cell_ijk(c)
        out = np.zeros((self.n_cells, self.dim, 2), dtype=np.int64)
        for a in range(self.dim):
            lo = [i, j, k]
            hi = [i.copy(), j.copy(), k.copy()]
            hi[a] = hi[a] + 1
            out[:, a, 0] = self.face_id(a, *lo)
            out[:, a, 1] = self.face_id(a, *hi)
        return out

    @property
    def cell_faces(self):
        return self._cell_faces

    def face_axis(self, e):
        return np.searchsorted(self.face_offset, e, side="right") - 1

    def face_cells(self):
        """(n_faces, 2) cell on the lower side and on the upper side (-1 if outside)."""
        fc = -np.ones((self.n_faces, 2), dtype=np.int64)
        cf = self._cell_faces
        for a in range(self.dim):
            fc[cf[:, a, 1], 0] = np.arange(self.n_cells)  # cell below the face
            fc[cf[:, a, 0], 1] = np.arange(self.n_cells)  # cell above the face
        return fc

    # ---- local matrices (Sec. 2, eqs. (a), (b)) --------------------------
    def cell_mass_block(self, c, a):
        """2x2 block of a(.,.) for cell c on its lower/upper a-faces."""
        h = self.grid.h[a]
        s = (h * h / self.vol) / self.perm[c, a]
        return s * np.array([[MASS_DIAG, MASS_OFF], [MASS_OFF, MASS_DIAG]])

    def assemble(self, cells, faces):
        """Matrices of a and b restricted to ``cells`` and to the face list
        ``faces`` (faces of those cells outside the list are dropped).

        Returns (A, B) as dense arrays: A is |faces| x |faces|, B is
        |cells| x |faces| with the sign convention of the module docstring.
        """
        pos = {int(e): n for n, e in enumerate(faces)}
        A = np.zeros((len(faces), len(faces)))
        B = np.zeros((len(cells), len(faces)))
        for r, c in enumerate(cells):
            for a in range(self.dim):
                blk = self.cell_mass_block(c, a)
                ids = [pos.get(int(self._cell_faces[c, a, s]), -1) for s in (0, 1)]
                for s1 in range(2):
                    if ids[s1] < 0:
                        continue
                    B[r, ids[s1]] += 1.0 if s1 == 0 else -1.0
                    for s2 in range(2):
                        if ids[s2] >= 0:
                            A[ids[s1], ids[s2]] += blk[s1, s2]
        return A, B

    def assemble_global_sparse(self):
        """Sparse global A (free faces) and B (cells x free faces)."""
        free_ids = np.nonzero(self.free)[0]
        fpos = -np.ones(self.n_faces, dtype=np.int64)
        fpos[free_ids] = np.arange(len(free_ids))
        rowsA, colsA, valsA = [], [], []
        rowsB, colsB, valsB = [], [], []
        for c in range(self.n_cells):
            for a in range(self.dim):
                blk = self.cell_mass_block(c, a)
                ids = [fpos[self._cell_faces[c, a, s]] for s in (0, 1)]
                for s1 in range(2):
                    if ids[s1] < 0:
                        continue
                    rowsB.append(c)
                    colsB.append(ids[s1])
                    valsB.append(1.0 if s1 == 0 else -1.0)
                    for s2 in range(2):
                        if ids[s2] >= 0:
                            rowsA.append(ids[s1])
                            colsA.append(ids[s2])
                            valsA.append(blk[s1, s2])
        nf = len(free_ids)
        A = sp.csr_matrix((valsA, (rowsA, colsA)), shape=(nf, nf))
        B = sp.csr_matrix((valsB, (rowsB, colsB)), shape=(self.n_cells, nf))
        return free_ids, A, B

    # ---- right-hand sides (Sec. 2, eq. (rhs); boundary reading) ----------
    def cell_rhs(self):
        """<f, q_c> = -int_c f for each cell."""
        return -self.f * self.vol

    def face_rhs(self):
        """Flux-equation right-hand side g per global face (pressure data)."""
        g = np.zeros(self.n_faces)
        fc = self.face_cells()
        d = np.nonzero(self.dirichlet)[0]
        # a boundary face with no cell above it sits on the maximum side
        on_max = fc[d, 1] < 0
        g[d] = np.where(on_max, -self.bc_value[d], self.bc_value[d])
        return g


def direct_solve(disc: Discretization):
    """Solve the assembled saddle-point system (Sec. 4, eq. (system)) with a
    sparse direct solver: the exact discrete solution used to pin the BDDC
    result.  Pure-flux problems fix the pressure constant by a zero-mean
    constraint (Q has zero mean, Sec. 2).

    Returns (flux over all global faces, pressure per cell).
    """
    free_ids, A, B = disc.assemble_global_sparse()
    g = disc.face_rhs()[free_ids]
    fc = disc.cell_rhs()
    nf, nc = A.shape[0], disc.n_cells
    pure_flux = not np.any(disc.dirichlet)
    if pure_flux:
        vol = np.full((1, nc), disc.vol)
        K = sp.bmat([[A, B.T, None], [B, None, sp.csr_matrix(vol.T)],
                     [None, sp.csr_matrix(vol), None]], format="csc")
        rhs = np.concatenate([g, fc, [0.0]])
    else:
        K = sp.bmat([[A, B.T], [B, None]], format="csc")
        rhs = np.concatenate([g, fc])
    sol = spla.spsolve(K, rhs)
    flux = np.zeros(disc.n_faces)
    flux[free_ids] = sol[:nf]
    return flux, sol[nf:nf + nc]


def residuals(disc: Discretization, flux, pressure):
    """Residuals of both block rows of eq. (system) for a candidate solution:
    (flux-equation residual over free faces, cellwise mass residual)."""
    free_ids, A, B = disc.assemble_global_sparse()
    u = flux[free_ids]
    r1 = disc.face_rhs()[free_ids] - (A @ u + B.T @ pressure)
    r2 = disc.cell_rhs() - B @ u
    return r1, r2

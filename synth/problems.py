"""Grids, permeability fields, partitions and forcing (inputs only).

Layout conventions shared by every consumer of these inputs:

* Cells are numbered lexicographically, ``c = i + nx*(j + ny*k)``.
* Faces are numbered axis-major: all x-faces, then all y-faces, then (3D)
  all z-faces.  Within axis ``a`` the face with lower corner index
  ``(i, j, k)`` (one more position along ``a`` than there are cells) is
  numbered lexicographically with the extended extent along ``a``.
* A flux value on a face is the total normal flux through it, positive in the
  +axis direction.
* Boundary-condition arrays have one entry per face: type ``-1`` for faces
  inside the domain, ``0`` for a prescribed normal flux (only zero, "no flow",
  is used), ``1`` for a prescribed pressure, with the value in ``bc_value``.
* ``f`` is the source density per unit volume in each cell (positive for
  injection), so the integral of ``f`` over cell ``c`` is ``f[c] * |c|``.
* In 2D the cells have unit thickness (``h[2] == 1``).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Grid", "Problem", "n_faces", "face_axis_counts", "box_partition",
    "irregular_box_partition", "lognormal_iid", "gaussian_field",
    "channelized_2d", "layered_3d", "subdomain_constant", "pressure_drop_bc",
    "directional_pressure_bc", "no_flow_bc", "corner_wells", "make_config",
]


@dataclasses.dataclass(frozen=True)
class Grid:
    dim: int
    n: tuple  # cells per axis (nx, ny, nz); nz == 1 in 2D
    h: tuple  # cell size per axis (hx, hy, hz); hz == 1 in 2D

    @property
    def n_cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def cell_volume(self) -> float:
        return float(self.h[0] * self.h[1] * self.h[2])


@dataclasses.dataclass
class Problem:
    name: str
    grid: Grid
    perm: np.ndarray        # (n_cells,) or (n_cells, dim), float64, > 0
    partition: np.ndarray   # (n_cells,) int32 subdomain id per cell
    bc_type: np.ndarray     # (n_faces,) int8
    bc_value: np.ndarray    # (n_faces,) float64
    f: np.ndarray           # (n_cells,) float64 source density


def face_axis_counts(grid: Grid):
    """Number of faces normal to each axis (len == dim)."""
    nx, ny, nz = grid.n
    counts = [(nx + 1) * ny * nz, nx * (ny + 1) * nz]
    if grid.dim == 3:
        counts.append(nx * ny * (nz + 1))
    return counts


def n_faces(grid: Grid) -> int:
    return int(sum(face_axis_counts(grid)))


def _boundary_face_lists(grid: Grid):
    """Global indices and face-centre coordinates of the boundary faces.

    Returns a list of (axis, side, face_ids, centres) with side 0 = min
    (coordinate 0), side 1 = max.
    """
    nx, ny, nz = grid.n
    hx, hy, hz = grid.h
    out = []
    offs = np.cumsum([0] + face_axis_counts(grid))
    for a in range(grid.dim):
        ext = [nx, ny, nz]
        ext[a] += 1
        for side in (0, 1):
            pos = 0 if side == 0 else ext[a] - 1
            idx = np.indices((ext[2], ext[1], ext[0])).reshape(3, -1)
            k, j, i = idx
            ijk = [i, j, k]
            sel = ijk[a] == pos
            i, j, k = i[sel], j[sel], k[sel]
            fid = offs[a] + i + ext[0] * (j + ext[1] * k)
            cx = (i + (0.0 if a == 0 else 0.5)) * hx
            cy = (j + (0.0 if a == 1 else 0.5)) * hy
            cz = (k + (0.0 if a == 2 else 0.5)) * hz
            out.append((a, side, fid.astype(np.int64), np.stack([cx, cy, cz], 1)))
    return out


def no_flow_bc(grid: Grid):
    nf = n_faces(grid)
    t = np.full(nf, -1, dtype=np.int8)
    v = np.zeros(nf)
    for _, _, fid, _ in _boundary_face_lists(grid):
        t[fid] = 0
    return t, v


def pressure_drop_bc(grid: Grid, p_left: float = 1.0, p_right: float = 0.0):
    """Pressure ``p_left`` on x = 0, ``p_right`` on x = L, no flow elsewhere."""
    t, v = no_flow_bc(grid)
    for a, side, fid, _ in _boundary_face_lists(grid):
        if a == 0:
            t[fid] = 1
            v[fid] = p_left if side == 0 else p_right
    return t, v


def directional_pressure_bc(grid: Grid, theta: float):
    """Pressure on the whole boundary, p = -(x cos(theta) + y sin(theta)) / L.

    L is the domain diagonal length; used for the serving stream's random
    pressure-drop direction.
    """
    nf = n_faces(grid)
    t = np.full(nf, -1, dtype=np.int8)
    v = np.zeros(nf)
    lx, ly = grid.n[0] * grid.h[0], grid.n[1] * grid.h[1]
    L = math.hypot(lx, ly)
    for _, _, fid, c in _boundary_face_lists(grid):
        t[fid] = 1
        v[fid] = -(c[:, 0] * math.cos(theta) + c[:, 1] * math.sin(theta)) / L
    return t, v


def corner_wells(grid: Grid, rate: float = 1.0):
    """Injection in the first corner cell, production in the opposite one."""
    f = np.zeros(grid.n_cells)
    vol = grid.cell_volume
    f[0] = rate / vol
    f[grid.n_cells - 1] = -rate / vol
    return f


def box_partition(grid: Grid, parts) -> np.ndarray:
    """Regular partition into ``parts`` = (px, py[, pz]) boxes of equal size
    (the last box along an axis takes any remainder)."""
    nx, ny, nz = grid.n
    parts = list(parts) + [1] * (3 - len(parts))
    ids = []
    for a, (n, p) in enumerate(zip((nx, ny, nz), parts)):
        size = n // p
        ids.append(np.minimum(np.arange(n) // size, p - 1))
    k, j, i = np.meshgrid(ids[2], ids[1], ids[0], indexing="ij")
    part = i + parts[0] * (j + parts[1] * k)
    return part.reshape(-1).astype(np.int32)


def _segments(n, rng, lo, hi):
    cuts = [0]
    while cuts[-1] < n:
        cuts.append(cuts[-1] + int(rng.integers(lo, hi + 1)))
    cuts[-1] = n
    if len(cuts) > 2 and cuts[-1] - cuts[-2] < lo:
        cuts.pop(-2)
    return np.array(cuts)


def irregular_box_partition(grid: Grid, seed: int, lo: int = 3, hi: int = 8):
    """Tensor-product box partition with seeded segment lengths in [lo, hi]
    per axis (a short last segment is merged into its neighbour)."""
    rng = np.random.default_rng(seed)
    ids, counts = [], []
    for a in range(3):
        n = grid.n[a]
        if a >= grid.dim:
            ids.append(np.zeros(n, dtype=np.int64))
            counts.append(1)
            continue
        cuts = _segments(n, rng, lo, hi)
        ids.append(np.searchsorted(cuts, np.arange(n), side="right") - 1)
        counts.append(len(cuts) - 1)
    k, j, i = np.meshgrid(ids[2], ids[1], ids[0], indexing="ij")
    part = i + counts[0] * (j + counts[1] * k)
    return part.reshape(-1).astype(np.int32)


def lognormal_iid(grid: Grid, seed: int, mean10: float = 0.0, sigma10: float = 1.0):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.normal(mean10, sigma10, grid.n_cells)


def gaussian_field(shape_zyx, corr_zyx, rng) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian field by separable Gaussian filtering
    of white noise (correlation lengths in cells, per axis)."""
    from scipy.ndimage import gaussian_filter

    w = rng.standard_normal(shape_zyx)
    g = gaussian_filter(w, sigma=corr_zyx, mode="wrap")
    g -= g.mean()
    s = g.std()
    return g / (s if s > 0 else 1.0)


def _channel_layer(nx, ny, rng, log10_field, drift=None):
    """Overwrite one (ny, nx) layer of log10 k with sinuous channels along y."""
    n_ch = int(rng.integers(6, 13))
    params = drift if drift is not None else []
    if drift is None:
        for _ in range(n_ch):
            params.append(dict(
                x0=rng.uniform(0, nx), A=rng.uniform(3, 12), lam=rng.uniform(40, 120),
                phi=rng.uniform(0, 2 * math.pi), width=int(rng.integers(3, 9))))
    y = np.arange(ny) + 0.5
    x = np.arange(nx) + 0.5
    for p in params:
        xc = p["x0"] + p["A"] * np.sin(2 * math.pi * y / p["lam"] + p["phi"])
        mask = np.abs(x[None, :] - xc[:, None]) <= 0.5 * p["width"]
        vals = rng.uniform(3.0, 4.0, size=(ny, nx))
        log10_field[mask] = vals[mask]
    return params


def channelized_2d(grid: Grid, seed: int) -> np.ndarray:
    """Fluvial-like 2D field: smooth background in [1e-3, 1] and 6-12 sinuous
    channels of width 3-8 cells at 1e3-1e4 (contrast about 1e7)."""
    nx, ny = grid.n[0], grid.n[1]
    rng = np.random.default_rng(seed)
    g = gaussian_field((ny, nx), (5.0, 5.0), rng)
    lo, hi = g.min(), g.max()
    log10k = -3.0 + 3.0 * (g - lo) / (hi - lo if hi > lo else 1.0)
    _channel_layer(nx, ny, rng, log10k)
    return 10.0 ** log10k.reshape(-1)


def layered_3d(grid: Grid, seed: int) -> np.ndarray:
    """3D field: ln k = 2.5 * Gaussian (correlation 4 x 4 x 1 cells) with the
    bottom third of the layers replaced by slowly drifting channel layers."""
    nx, ny, nz = grid.n
    rng = np.random.default_rng(seed)
    g = gaussian_field((nz, ny, nx), (1.0, 4.0, 4.0), rng)
    log10k = 2.5 * g / math.log(10.0)
    n_bot = nz // 3
    params = None
    for kz in range(nz - n_bot, nz):
        layer = log10k[kz]
        if params is None:
            params = _channel_layer(nx, ny, rng, layer)
        else:
            for p in params:
                p["x0"] += rng.normal(0.0, 0.5)
                p["phi"] += rng.normal(0.0, 0.05)
            _channel_layer(nx, ny, rng, layer, drift=params)
    return 10.0 ** log10k.reshape(-1)


def subdomain_constant(partition: np.ndarray, seed: int, lo10: float = -3.0, hi10: float = 3.0,
                       n_comp: int = 1) -> np.ndarray:
    """Permeability constant inside every subdomain (jumps aligned with the
    subdomain interfaces, the setting of the paper's stiffness-scaling test):
    log10 k ~ U[lo10, hi10] per subdomain (and per axis when n_comp > 1)."""
    rng = np.random.default_rng(seed)
    n_sub = int(partition.max()) + 1
    vals = 10.0 ** rng.uniform(lo10, hi10, (n_sub, n_comp))
    k = vals[partition]
    return np.ascontiguousarray(k[:, 0] if n_comp == 1 else k)


def make_config(name: str, seed: int | None = None) -> Problem:
    """Named seeded workloads.

    c1      16 x 16 unit square, 4 x 4 subdomains, iid log-normal k
            (log10 mean 0, sigma 1), unit pressure drop left to right.
    c2      60 x 220 cells of 20 x 10 ft, 6 x 22 subdomains of 10 x 10,
            channelized k (contrast ~1e7), unit pressure drop along x.
    c3      60 x 220 x 85 cells of 20 x 10 x 2 ft, 12 x 44 x 17 subdomains
            of 5^3, layered 3D field.
    c4      as c3 with a seeded irregular box partition (3-8 cells per axis).
    pin2d   60 x 220 cells of 20 x 10 ft, k = 1, 6 x 22 subdomains,
            corner wells (the paper's homogeneous 2D case).
    pin3d   30^3 cells of 20 x 10 x 2 ft, k = 1, 3 x 3 x 3 subdomains,
            corner wells (the paper's homogeneous 3D case).
    tiny3d  4^3 unit cube, 2 x 2 x 2 subdomains, iid log-normal k,
            pressure drop.
    """
    if name == "c1":
        s = 1901 if seed is None else seed
        g = Grid(2, (16, 16, 1), (1 / 16, 1 / 16, 1.0))
        perm = lognormal_iid(g, s)
        part = box_partition(g, (4, 4))
        t, v = pressure_drop_bc(g)
        f = np.zeros(g.n_cells)
    elif name == "c2":
        s = 2090 if seed is None else seed
        g = Grid(2, (60, 220, 1), (20.0, 10.0, 1.0))
        perm = channelized_2d(g, s)
        part = box_partition(g, (6, 22))
        t, v = pressure_drop_bc(g)
        f = np.zeros(g.n_cells)
    elif name in ("c3", "c4"):
        s = (3085 if name == "c3" else 4085) if seed is None else seed
        g = Grid(3, (60, 220, 85), (20.0, 10.0, 2.0))
        perm = layered_3d(g, s)
        part = box_partition(g, (12, 44, 17)) if name == "c3" else irregular_box_partition(g, s)
        t, v = pressure_drop_bc(g)
        f = np.zeros(g.n_cells)
    elif name == "pin2d":
        g = Grid(2, (60, 220, 1), (20.0, 10.0, 1.0))
        perm = np.ones(g.n_cells)
        part = box_partition(g, (6, 22))
        t, v = no_flow_bc(g)
        f = corner_wells(g)
    elif name == "pin3d":
        g = Grid(3, (30, 30, 30), (20.0, 10.0, 2.0))
        perm = np.ones(g.n_cells)
        part = box_partition(g, (3, 3, 3))
        t, v = no_flow_bc(g)
        f = corner_wells(g)
    elif name == "tiny3d":
        s = 43 if seed is None else seed
        g = Grid(3, (4, 4, 4), (0.25, 0.25, 0.25))
        perm = lognormal_iid(g, s)
        part = box_partition(g, (2, 2, 2))
        t, v = pressure_drop_bc(g)
        f = np.zeros(g.n_cells)
    else:
        raise ValueError(f"unknown config {name!r}")
    return Problem(name, g, np.ascontiguousarray(perm, dtype=np.float64),
                   part.astype(np.int32), t, v, f)


def serving_request(request_id: int, base_seed: int = 5000) -> Problem:
    """One request of the serving stream: a channelized 2D field of
    nx in {30,40,50,60} by ny in {110,...,220} cells (20 x 10 ft), 10 x 10
    subdomains, pressure on the whole boundary with a random direction."""
    rng = np.random.default_rng(base_seed + request_id)
    nx = int(rng.choice([30, 40, 50, 60]))
    ny = int(rng.choice(np.arange(110, 221, 10)))
    g = Grid(2, (nx, ny, 1), (20.0, 10.0, 1.0))
    perm = channelized_2d(g, base_seed * 7 + request_id)
    part = box_partition(g, (nx // 10, ny // 10))
    t, v = directional_pressure_bc(g, float(rng.uniform(0, 2 * math.pi)))
    return Problem(f"req{request_id}", g, perm, part, t, v, np.zeros(g.n_cells))

"""Seeded synthetic inputs: face-list meshes, discrete velocity grids, initial fields.

This module builds the *inputs* of a UGKS run and nothing else: mesh geometry
(cell volumes and centroids, face areas, unit normals and centroids, owner /
neighbour lists), discrete velocity sets with their quadrature weights, and
primitive initial fields (rho, U, T).  It contains none of the scheme's
arithmetic (no Maxwellians, fluxes, reconstructions or moments), so it can be
shared by the CUDA path and by the FP64 oracle without coupling them.

Conventions (shared by every consumer):
  * ``face_neighbor[f] >= 0`` is an interior face; ``face_neighbor[f] < 0``
    encodes boundary condition ``bc[-face_neighbor[f] - 1]``.
  * ``face_normal[f]`` is the unit normal pointing from the owner cell to the
    neighbour cell (outward from the owner on boundary faces).
  * ``face_shift[f]`` is the translation to add to the neighbour's centroid as
    seen across face ``f`` (non-zero only on periodic faces).
  * Velocity grids are tensor products with the first axis fastest, so a block
    of ``n_x`` consecutive velocities is one line along u_x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

BC_WALL = 1       # diffuse-reflection isothermal wall (Sec. 2.1, Eq. 36-38)
BC_FARFIELD = 2   # ghost state fixed to the boundary's (rho, U, T)
BC_OUTFLOW = 3    # ghost state copied from the interior cell


@dataclasses.dataclass
class BC:
    type: int
    rho: float = 1.0
    u: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    T: float = 1.0


@dataclasses.dataclass
class Mesh:
    dim: int
    cell_volume: np.ndarray      # [Nc] f64
    cell_centroid: np.ndarray    # [Nc, dim] f64
    face_owner: np.ndarray       # [Nf] i64
    face_neighbor: np.ndarray    # [Nf] i64
    face_area: np.ndarray        # [Nf] f64
    face_normal: np.ndarray      # [Nf, dim] f64
    face_centroid: np.ndarray    # [Nf, dim] f64
    face_shift: np.ndarray       # [Nf, dim] f64
    bc: List[BC]
    name: str = ""

    @property
    def n_cells(self) -> int:
        return int(self.cell_volume.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.face_area.shape[0])

    def closure_residual(self) -> float:
        """max_i |sum_f sigma S n| / sum_f S  (zero for a closed cell)."""
        acc = np.zeros((self.n_cells, self.dim))
        tot = np.zeros(self.n_cells)
        sn = self.face_area[:, None] * self.face_normal
        np.add.at(acc, self.face_owner, sn)
        np.add.at(tot, self.face_owner, self.face_area)
        inner = self.face_neighbor >= 0
        np.add.at(acc, self.face_neighbor[inner], -sn[inner])
        np.add.at(tot, self.face_neighbor[inner], self.face_area[inner])
        return float(np.max(np.linalg.norm(acc, axis=1) / tot))


@dataclasses.dataclass
class VelocityGrid:
    u: np.ndarray        # [Nv, dim] f64
    weight: np.ndarray   # [Nv] f64
    axes: Optional[List[np.ndarray]] = None   # 1-D axes if a tensor grid (first fastest)

    @property
    def n_v(self) -> int:
        return int(self.weight.shape[0])

    @property
    def dim(self) -> int:
        return int(self.u.shape[1])


# ----------------------------------------------------------------------------
# Velocity grids
# ----------------------------------------------------------------------------

def _tensor(axes: Sequence[np.ndarray], weights: Sequence[np.ndarray]) -> VelocityGrid:
    dim = len(axes)
    grids = np.meshgrid(*axes, indexing="ij")
    wgrids = np.meshgrid(*weights, indexing="ij")
    # first axis fastest: transpose so that axis 0 varies fastest in C order
    order = tuple(reversed(range(dim)))
    u = np.stack([g.transpose(order).reshape(-1) for g in grids], axis=1)
    w = np.ones(u.shape[0])
    for wg in wgrids:
        w = w * wg.transpose(order).reshape(-1)
    return VelocityGrid(u=np.ascontiguousarray(u), weight=w,
                        axes=[np.asarray(a, dtype=np.float64) for a in axes])


def midpoint_grid(n, lo: float, hi: float, dim: int) -> VelocityGrid:
    """Composite midpoint (open Newton-Cotes) tensor grid on [lo, hi]^dim.

    Node i of each axis sits at the centre of velocity cell i, and the weight is
    the velocity-cell volume (the paper's omega_k, Sec. 2.1, Eq. 22)."""
    ns = [n] * dim if np.isscalar(n) else list(n)
    axes, ws = [], []
    for m in ns:
        d = (hi - lo) / m
        axes.append(lo + (np.arange(m) + 0.5) * d)
        ws.append(np.full(m, d))
    return _tensor(axes, ws)


def gauss_hermite_grid(n: int, umax: float, dim: int) -> VelocityGrid:
    """Scaled Gauss-Hermite tensor grid of the cavity test (Sec. 3.1, Eq. 65-67).

    Roots xi_i of the physicists' Hermite polynomial H_n are scaled by
    s = umax / max|xi_i|; the 1-D weight is s * w_i^GH * exp(xi_i^2)."""
    xi, wgh = np.polynomial.hermite.hermgauss(n)
    s = umax / np.max(np.abs(xi))
    v = s * xi
    w = s * wgh * np.exp(xi ** 2)
    return _tensor([v] * dim, [w] * dim)


# ----------------------------------------------------------------------------
# Cartesian face-list meshes (cavity, periodic boxes, strips)
# ----------------------------------------------------------------------------

def cartesian_mesh(shape: Sequence[int], lo: Sequence[float], hi: Sequence[float],
                   sides: Dict[str, object], bcs: List[BC], name: str = "") -> Mesh:
    """Uniform Cartesian mesh in 1, 2 or 3 dimensions, emitted as a face list.

    ``sides`` maps 'x-','x+','y-','y+','z-','z+' to a bc index, or to the
    string 'periodic' on both ends of an axis."""
    dim = len(shape)
    shape = [int(s) for s in shape]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    h = (hi - lo) / np.asarray(shape)
    ncell = int(np.prod(shape))
    idx = np.arange(ncell).reshape(list(reversed(shape)))  # [nz][ny][nx]
    idx = idx.transpose(list(reversed(range(dim))))         # idx[i][j][k]
    centers = []
    for a in range(dim):
        centers.append(lo[a] + (np.arange(shape[a]) + 0.5) * h[a])
    cc = np.stack(np.meshgrid(*centers, indexing="ij"), axis=-1)  # [nx,ny,nz,dim]
    cell_centroid = np.zeros((ncell, dim))
    cell_centroid[idx.reshape(-1)] = cc.reshape(-1, dim)
    cell_volume = np.full(ncell, float(np.prod(h)))

    owners, neigh, areas, normals, fcent, shifts = [], [], [], [], [], []
    names = "xyz"
    for a in range(dim):
        area = float(np.prod([h[b] for b in range(dim) if b != a])) if dim > 1 else 1.0
        e = np.zeros(dim)
        e[a] = 1.0
        lo_key, hi_key = names[a] + "-", names[a] + "+"
        periodic = sides.get(lo_key) == "periodic"
        # interior planes between slab s and s+1
        for s in range(shape[a] - 1):
            sl_o = [slice(None)] * dim
            sl_n = [slice(None)] * dim
            sl_o[a] = s
            sl_n[a] = s + 1
            o = idx[tuple(sl_o)].reshape(-1)
            nb = idx[tuple(sl_n)].reshape(-1)
            owners.append(o)
            neigh.append(nb)
            areas.append(np.full(o.size, area))
            normals.append(np.tile(e, (o.size, 1)))
            fc = cell_centroid[o].copy()
            fc[:, a] = lo[a] + (s + 1) * h[a]
            fcent.append(fc)
            shifts.append(np.zeros((o.size, dim)))
        sl_first = [slice(None)] * dim
        sl_last = [slice(None)] * dim
        sl_first[a] = 0
        sl_last[a] = shape[a] - 1
        first = idx[tuple(sl_first)].reshape(-1)
        last = idx[tuple(sl_last)].reshape(-1)
        if periodic:
            assert sides.get(hi_key) == "periodic"
            owners.append(last)
            neigh.append(first)
            areas.append(np.full(last.size, area))
            normals.append(np.tile(e, (last.size, 1)))
            fc = cell_centroid[last].copy()
            fc[:, a] = hi[a]
            fcent.append(fc)
            sh = np.zeros((last.size, dim))
            sh[:, a] = hi[a] - lo[a]
            shifts.append(sh)
        else:
            for cells, key, sign, plane in ((first, lo_key, -1.0, lo[a]), (last, hi_key, 1.0, hi[a])):
                bid = int(sides[key])
                owners.append(cells)
                neigh.append(np.full(cells.size, -(bid + 1), dtype=np.int64))
                areas.append(np.full(cells.size, area))
                normals.append(np.tile(sign * e, (cells.size, 1)))
                fc = cell_centroid[cells].copy()
                fc[:, a] = plane
                fcent.append(fc)
                shifts.append(np.zeros((cells.size, dim)))
    return Mesh(dim=dim, cell_volume=cell_volume, cell_centroid=cell_centroid,
                face_owner=np.concatenate(owners).astype(np.int64),
                face_neighbor=np.concatenate(neigh).astype(np.int64),
                face_area=np.concatenate(areas), face_normal=np.concatenate(normals),
                face_centroid=np.concatenate(fcent), face_shift=np.concatenate(shifts),
                bc=list(bcs), name=name)


def cavity_mesh(n: int = 32, lid_speed: float = 0.14606, T_wall: float = 1.0) -> Mesh:
    """2-D lid-driven cavity on [0,1]^2: n x n quads, 4n wall faces.

    bc 0 is the moving lid (y = 1) with wall velocity (lid_speed, 0); bc 1 the
    three stationary walls.  Both are isothermal at T_wall."""
    bcs = [BC(BC_WALL, 1.0, (lid_speed, 0.0, 0.0), T_wall), BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_wall)]
    return cartesian_mesh((n, n), (0.0, 0.0), (1.0, 1.0),
                          {"x-": 1, "x+": 1, "y-": 1, "y+": 0}, bcs, name=f"cavity{n}x{n}")


def periodic_box(shape: Sequence[int], length: Sequence[float] = None) -> Mesh:
    dim = len(shape)
    length = [1.0] * dim if length is None else list(length)
    sides = {}
    for a in range(dim):
        sides["xyz"[a] + "-"] = "periodic"
        sides["xyz"[a] + "+"] = "periodic"
    return cartesian_mesh(shape, [0.0] * dim, length, sides, [], name="periodic" + "x".join(map(str, shape)))


# ----------------------------------------------------------------------------
# Unstructured simplex meshes (tetrahedra around a sphere, triangles around a cylinder)
# ----------------------------------------------------------------------------

def _fibonacci_sphere(n: int, rng: np.random.Generator) -> np.ndarray:
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    theta = math.pi * (1.0 + 5.0 ** 0.5) * i
    p = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)
    # random rotation so that successive shells are not aligned
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return p @ q


def _simplex_faces(simplices: np.ndarray, points: np.ndarray, dim: int):
    """Face list of a simplicial complex: (owner, neighbour or -1, vertices)."""
    ns = simplices.shape[0]
    nv = dim + 1
    local = [[v for v in range(nv) if v != w] for w in range(nv)]
    tri = np.concatenate([simplices[:, l] for l in local], axis=0)     # [nv*ns, dim]
    cell = np.tile(np.arange(ns), nv)
    key = np.sort(tri, axis=1)
    _, inv, counts = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.reshape(-1)
    order = np.argsort(inv, kind="stable")
    inv_sorted = inv[order]
    starts = np.searchsorted(inv_sorted, np.arange(counts.size))
    owner = cell[order[starts]]
    verts = tri[order[starts]]
    neighbor = np.full(counts.size, -1, dtype=np.int64)
    two = counts == 2
    neighbor[two] = cell[order[starts[two] + 1]]
    if np.any(counts > 2):
        raise ValueError("non-manifold simplex complex")
    return owner.astype(np.int64), neighbor, verts


def _simplex_geometry(points, simplices, dim):
    v = points[simplices]                       # [ns, dim+1, dim]
    cent = v.mean(axis=1)
    mat = v[:, 1:, :] - v[:, :1, :]
    vol = np.abs(np.linalg.det(mat)) / math.factorial(dim)
    return cent, vol


def _face_geometry(points, verts, owner_centroid, dim):
    fv = points[verts]                          # [nf, dim, dim]
    fc = fv.mean(axis=1)
    if dim == 3:
        nrm = np.cross(fv[:, 1] - fv[:, 0], fv[:, 2] - fv[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
    else:
        t = fv[:, 1] - fv[:, 0]
        nrm = np.stack([t[:, 1], -t[:, 0]], axis=1)
        area = np.linalg.norm(nrm, axis=1)
    nrm = nrm / np.linalg.norm(nrm, axis=1)[:, None]
    flip = np.einsum("ij,ij->i", nrm, fc - owner_centroid) < 0
    nrm[flip] *= -1.0
    return fc, area, nrm


def _assemble_simplex_mesh(points, simplices, keep, dim, classify, bcs, name):
    from scipy.spatial import Delaunay  # noqa: F401  (scipy is required by the generators)
    simp = simplices[keep]
    cent, vol = _simplex_geometry(points, simp, dim)
    owner, neighbor, verts = _simplex_faces(simp, points, dim)
    fc, area, nrm = _face_geometry(points, verts, cent[owner], dim)
    bnd = neighbor < 0
    neighbor[bnd] = -(classify(fc[bnd]) + 1)
    return Mesh(dim=dim, cell_volume=vol, cell_centroid=cent, face_owner=owner,
                face_neighbor=neighbor, face_area=area, face_normal=nrm, face_centroid=fc,
                face_shift=np.zeros_like(fc), bc=bcs, name=name)


def _size_search(build, target: int, dim: int, scale0: float = 1.0, tol: float = 0.05, max_iter: int = 12):
    """Finds the spacing scale whose mesh has target +- tol cells, using the
    power law cells ~ scale^-dim (secant steps in log-log space from scale0)."""
    scale = scale0
    P, simp, keep = build(scale)
    n = int(keep.sum())
    expo = float(dim)
    prev = None
    for _ in range(max_iter):
        if abs(n - target) <= tol * target:
            break
        if prev is not None and prev[1] != n and prev[0] != scale:
            e = -math.log(n / prev[1]) / math.log(scale / prev[0])
            if 0.5 * dim <= e <= 2.0 * dim:
                expo = e
        new_scale = scale * (n / target) ** (1.0 / expo)
        prev = (scale, n)
        scale = new_scale
        P, simp, keep = build(scale)
        n = int(keep.sum())
    return P, simp, keep


def sphere_tet_mesh(target_cells: int = 100_000, seed: int = 2, mach: float = 5.0,
                    T_wall: Optional[float] = None, gamma: float = 5.0 / 3.0) -> Mesh:
    """Tetrahedral mesh around a unit sphere in the box [-4,8] x [-5,5]^2.

    Points: Fibonacci shells graded away from the body (spacing proportional to
    0.04 + 0.12 (r - 1)) plus lattices on the box faces; Delaunay
    triangulation; tetrahedra whose centroid lies inside r < 1 are removed.
    The overall spacing scale is bisected until the cell count is within 5% of
    ``target_cells``.  bc 0: diffuse wall at T_wall (stagnation temperature by
    default); bc 1: far field (rho=1, U=(Ma sqrt(gamma/2), 0, 0), T=1); bc 2:
    outflow at x = 8."""
    from scipy.spatial import Delaunay
    lo = np.array([-4.0, -5.0, -5.0])
    hi = np.array([8.0, 5.0, 5.0])
    u_inf = mach * math.sqrt(gamma / 2.0)
    if T_wall is None:
        T_wall = 1.0 + 0.5 * (gamma - 1.0) * mach ** 2
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_wall), BC(BC_FARFIELD, 1.0, (u_inf, 0.0, 0.0), 1.0),
           BC(BC_OUTFLOW, 1.0, (u_inf, 0.0, 0.0), 1.0)]
    rmax = float(np.linalg.norm(np.maximum(np.abs(lo), np.abs(hi))))

    def build(scale):
        rng = np.random.default_rng(seed)
        pts = []
        r = 1.0
        while r < rmax:
            hh = scale * (0.04 + 0.12 * (r - 1.0))
            n = max(12, int(round(4.0 * math.pi * r * r / (hh * hh))))
            p = r * _fibonacci_sphere(n, rng)
            inside = np.all((p > lo + 0.35 * hh) & (p < hi - 0.35 * hh), axis=1)
            pts.append(p[inside])
            r += hh
        # lattices on the six box faces, spacing of the local shell
        for a in range(3):
            for plane in (lo[a], hi[a]):
                hh = scale * (0.04 + 0.12 * (max(abs(plane), 1.0) + 1.0))
                others = [b for b in range(3) if b != a]
                g0 = np.linspace(lo[others[0]], hi[others[0]], int(np.ceil((hi[others[0]] - lo[others[0]]) / hh)) + 1)
                g1 = np.linspace(lo[others[1]], hi[others[1]], int(np.ceil((hi[others[1]] - lo[others[1]]) / hh)) + 1)
                G0, G1 = np.meshgrid(g0, g1, indexing="ij")
                p = np.zeros((G0.size, 3))
                p[:, a] = plane
                p[:, others[0]] = G0.reshape(-1)
                p[:, others[1]] = G1.reshape(-1)
                pts.append(p)
        P = np.unique(np.round(np.concatenate(pts), 12), axis=0)
        tri = Delaunay(P, qhull_options="Qbb Qc Qz Q12")
        simp = tri.simplices.astype(np.int64)
        cent = P[simp].mean(axis=1)
        keep = np.linalg.norm(cent, axis=1) > 1.0
        _, vol = _simplex_geometry(P, simp, 3)
        keep &= vol > 1e-14
        return P, simp, keep

    P, simp, keep = _size_search(build, target_cells, dim=3,
                                 scale0=1.6133 * (103387.0 / target_cells) ** (1.0 / 3.0))

    def classify(fc):
        out = np.full(fc.shape[0], 1, dtype=np.int64)
        out[np.linalg.norm(fc, axis=1) < 1.5] = 0
        out[np.abs(fc[:, 0] - hi[0]) < 1e-9] = 2
        return out

    return _assemble_simplex_mesh(P, simp, keep, 3, classify, bcs, name=f"sphere_tet{int(keep.sum())}")


def box_tet_mesh(n_inner: int = 2, seed: int = 7, bcs: Optional[List[BC]] = None) -> Mesh:
    """Delaunay tetrahedra of the unit cube's corners and ``n_inner`` seeded
    interior points (a few cells with skewed, non-orthogonal neighbours).
    Boundary faces: x = 0 -> bc 0, x = 1 -> bc 1, the others -> bc 2
    (default: far field, outflow, wall)."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    corners = np.array([[x, y, z] for x in (0.0, 1.0) for y in (0.0, 1.0) for z in (0.0, 1.0)])
    pts = np.vstack([corners, rng.uniform(0.2, 0.8, (n_inner, 3))])
    tri = Delaunay(pts)
    if bcs is None:
        bcs = [BC(BC_FARFIELD, 1.05, (0.25, 0.0, 0.1), 1.1), BC(BC_OUTFLOW), BC(BC_WALL, 1.0, (0.0, 0.1, 0.0), 1.2)]

    def classify(fc):
        return np.where(fc[:, 0] < 1e-9, 0, np.where(fc[:, 0] > 1.0 - 1e-9, 1, 2))
    return _assemble_simplex_mesh(pts, tri.simplices, np.ones(len(tri.simplices), bool), 3, classify, bcs,
                                  name=f"box_tet{len(tri.simplices)}")


def cylinder_tri_mesh(target_cells: int = 10_000, seed: int = 4, mach: float = 3.0,
                      T_wall: Optional[float] = None, gamma: float = 5.0 / 3.0, radius: float = 0.5,
                      lateral: str = "outflow") -> Mesh:
    """Triangle mesh around a cylinder of the given radius in [-4,8] x [-5,5].

    Graded circular rings (spacing proportional to 0.02 + 0.1 (r - R)), lattices
    on the box edges, Delaunay, triangles inside r < R removed.  bc 0 wall,
    bc 1 far field (the inflow edge x = -4, and the edges y = +-5 when
    ``lateral`` is "farfield"), bc 2 outflow at x = 8 and, by default, at
    y = +-5: the bow shock of a supersonic stream leaves through the lateral
    edges, and a free-stream ghost state there holds the post-shock gas
    against the free stream (above Ma ~7 on these meshes the cells where the
    shock meets the edges went to T ~ 0)."""
    from scipy.spatial import Delaunay
    lo = np.array([-4.0, -5.0])
    hi = np.array([8.0, 5.0])
    u_inf = mach * math.sqrt(gamma / 2.0)
    if T_wall is None:
        T_wall = 1.0 + 0.5 * (gamma - 1.0) * mach ** 2
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_wall), BC(BC_FARFIELD, 1.0, (u_inf, 0.0, 0.0), 1.0),
           BC(BC_OUTFLOW, 1.0, (u_inf, 0.0, 0.0), 1.0)]
    rmax = float(np.linalg.norm(np.maximum(np.abs(lo), np.abs(hi))))

    def build(scale):
        rng = np.random.default_rng(seed)
        pts = []
        r = radius
        while r < rmax:
            hh = scale * (0.02 + 0.1 * (r - radius))
            n = max(8, int(round(2.0 * math.pi * r / hh)))
            th = 2.0 * math.pi * (np.arange(n) + rng.uniform()) / n
            p = r * np.stack([np.cos(th), np.sin(th)], axis=1)
            inside = np.all((p > lo + 0.35 * hh) & (p < hi - 0.35 * hh), axis=1)
            pts.append(p[inside])
            r += hh
        for a in range(2):
            for plane in (lo[a], hi[a]):
                hh = scale * (0.02 + 0.1 * (max(abs(plane), radius) - radius))
                b = 1 - a
                g = np.linspace(lo[b], hi[b], int(np.ceil((hi[b] - lo[b]) / hh)) + 1)
                p = np.zeros((g.size, 2))
                p[:, a] = plane
                p[:, b] = g
                pts.append(p)
        P = np.unique(np.round(np.concatenate(pts), 12), axis=0)
        tri = Delaunay(P, qhull_options="Qbb Qc Qz Q12")
        simp = tri.simplices.astype(np.int64)
        cent = P[simp].mean(axis=1)
        keep = np.linalg.norm(cent, axis=1) > radius
        _, vol = _simplex_geometry(P, simp, 2)
        keep &= vol > 1e-14
        return P, simp, keep

    P, simp, keep = _size_search(build, target_cells, dim=2)

    def classify(fc):
        out = np.full(fc.shape[0], 1, dtype=np.int64)
        out[np.linalg.norm(fc, axis=1) < radius + 0.5 * (radius * 0.2 + 0.05)] = 0
        out[np.abs(fc[:, 0] - hi[0]) < 1e-9] = 2
        if lateral == "outflow":
            out[(np.abs(fc[:, 1] - lo[1]) < 1e-9) | (np.abs(fc[:, 1] - hi[1]) < 1e-9)] = 2
        elif lateral != "farfield":
            raise ValueError("lateral must be 'outflow' or 'farfield'")
        return out

    return _assemble_simplex_mesh(P, simp, keep, 2, classify, bcs, name=f"cylinder_tri{int(keep.sum())}")


# ----------------------------------------------------------------------------
# Initial primitive fields (rho, U, T) -- seeded
# ----------------------------------------------------------------------------

def uniform_primitives(mesh: Mesh, rho: float = 1.0, U=(0.0, 0.0, 0.0), T: float = 1.0) -> np.ndarray:
    """[Nc, dim+2] array of (rho, U_1..U_dim, T)."""
    out = np.zeros((mesh.n_cells, mesh.dim + 2))
    out[:, 0] = rho
    out[:, 1:1 + mesh.dim] = np.asarray(U, dtype=np.float64)[:mesh.dim]
    out[:, -1] = T
    return out


def cylinder_potential_primitives(mesh: Mesh, u_inf: float, radius: float = 0.5, rho: float = 1.0,
                                  T: float = 1.0) -> np.ndarray:
    """Start-up field for a cylinder of the given radius at the origin in a
    stream u_inf along x: the velocity of incompressible potential flow,
    u - i v = u_inf (1 - R^2 / z^2), scaled down wherever its speed exceeds
    u_inf (so that it stays inside a velocity grid sized for the free
    stream), with uniform rho and T.  It is tangential at the wall and zero at
    both stagnation points, so, unlike a uniform free stream, it does not pull
    the gas away from the rear of the body at the first step (a uniform start
    empties the cells behind the cylinder to ~1e-6 of the free-stream
    density)."""
    x = mesh.cell_centroid[:, 0]
    y = mesh.cell_centroid[:, 1]
    r2 = x * x + y * y
    R2 = radius * radius
    u = u_inf * (1.0 - R2 * (x * x - y * y) / (r2 * r2))
    v = -u_inf * 2.0 * R2 * x * y / (r2 * r2)
    speed = np.sqrt(u * u + v * v)
    scale = np.minimum(1.0, u_inf / np.maximum(speed, 1e-300))
    out = np.zeros((mesh.n_cells, mesh.dim + 2))
    out[:, 0] = rho
    out[:, 1] = u * scale
    out[:, 2] = v * scale
    out[:, -1] = T
    return out


def smooth_random_primitives(mesh: Mesh, seed: int, amp: float = 0.1, modes: int = 3,
                             rho0: float = 1.0, U0=(0.0, 0.0, 0.0), T0: float = 1.0,
                             length: Optional[Sequence[float]] = None) -> np.ndarray:
    """Smooth seeded perturbation of a uniform state: sum of random Fourier modes
    (integer wave numbers on ``length`` so that the field is periodic there)."""
    rng = np.random.default_rng(seed)
    x = mesh.cell_centroid
    dim = mesh.dim
    L = np.ones(dim) if length is None else np.asarray(length, dtype=np.float64)
    prim = uniform_primitives(mesh, rho0, U0, T0)
    for comp in range(dim + 2):
        field = np.zeros(mesh.n_cells)
        for _ in range(modes):
            kv = rng.integers(-2, 3, size=dim)
            if not np.any(kv):
                kv[0] = 1
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            field += a * np.sin(2 * math.pi * (x / L) @ kv + ph)
        field *= amp / modes
        if comp == 0:
            prim[:, 0] *= 1.0 + field
        elif comp == dim + 1:
            prim[:, -1] *= 1.0 + field
        else:
            prim[:, comp] += field
    return prim


# ----------------------------------------------------------------------------
# Gas / run parameters (plain configuration; the scheme's arithmetic lives in
# the CUDA library and, independently, in the oracle)
# ----------------------------------------------------------------------------

LIMITERS = {"none": 0, "venkatakrishnan": 1, "barth_jespersen": 2}
MODELS = {"bgk": 0, "shakhov": 1}


def mu_ref_from_kn(kn: float, omega: float, alpha: float = 1.0) -> float:
    """Reference viscosity of the variable-hard-sphere model for a Knudsen
    number defined with the unit length, rho = 1 and sqrt(2RT) = 1 (Bird's
    mean-free-path relation; alpha = 1 for VHS)."""
    return 5.0 * (alpha + 1.0) * (alpha + 2.0) * math.sqrt(math.pi) / (
        4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega)) * kn


@dataclasses.dataclass
class Gas:
    K: int = 0                      # internal degrees of freedom
    model: str = "bgk"              # "bgk" | "shakhov"
    Pr: float = 1.0
    omega: float = 0.81             # viscosity exponent, mu = mu_ref T^omega
    mu_ref: float = 0.05
    cfl: float = 0.8
    dt: float = 0.0                 # > 0 overrides the CFL time step
    limiter: str = "venkatakrishnan"
    venkat_K: float = 5.0
    shock_tau_fix: bool = False


def prim_to_conservative(prim: np.ndarray, dim: int, K: int) -> np.ndarray:
    """(rho, U, T) -> (rho, rho U, rho E) with R = 1/2 (rho E = rho|U|^2/2 + (K+3) rho T / 4).

    This is the definition of the conservative variables, used by callers to
    build W_init from a primitive field."""
    W = np.zeros_like(prim)
    rho = prim[:, 0]
    U = prim[:, 1:1 + dim]
    T = prim[:, -1]
    W[:, 0] = rho
    W[:, 1:1 + dim] = rho[:, None] * U
    W[:, -1] = 0.5 * rho * np.sum(U * U, axis=1) + (K + 3) * rho * T / 4.0
    return W


def submesh(mesh: Mesh, seeds, rings: int):
    """Cells within ``rings`` face hops of ``seeds``, as a closed mesh.

    Faces to cells outside the patch become faces of an added outflow boundary
    condition (flipped so that the owner is inside).  Returns (cells, mesh)
    where ``cells`` are the original indices in patch order."""
    nb = [[] for _ in range(mesh.n_cells)]
    for o, n in zip(mesh.face_owner, mesh.face_neighbor):
        if n >= 0:
            nb[o].append(n)
            nb[n].append(o)
    cells = set(int(c) for c in seeds)
    frontier = set(cells)
    for _ in range(rings):
        new = {j for c in frontier for j in nb[c]} - cells
        cells |= new
        frontier = new
    cells = np.array(sorted(cells), dtype=np.int64)
    local = -np.ones(mesh.n_cells, dtype=np.int64)
    local[cells] = np.arange(cells.size)
    inside = local >= 0
    own, nei = mesh.face_owner, mesh.face_neighbor
    keep = inside[own] | ((nei >= 0) & inside[np.maximum(nei, 0)])
    fo, fn = own[keep], nei[keep]
    nrm = mesh.face_normal[keep].copy()
    cen = mesh.face_centroid[keep].copy()
    shift = mesh.face_shift[keep].copy()
    out_bc = len(mesh.bc)
    new_own = np.empty(fo.size, dtype=np.int64)
    new_nei = np.empty(fo.size, dtype=np.int64)
    for t in range(fo.size):
        o, n = fo[t], fn[t]
        if inside[o]:
            new_own[t] = local[o]
            if n < 0:
                new_nei[t] = n
            elif inside[n]:
                new_nei[t] = local[n]
            else:
                new_nei[t] = -(out_bc + 1)
                shift[t] = 0.0
        else:                                      # neighbour inside, owner outside: flip
            new_own[t] = local[n]
            new_nei[t] = -(out_bc + 1)
            nrm[t] = -nrm[t]
            cen[t] = cen[t] - shift[t]
            shift[t] = 0.0
    return cells, Mesh(dim=mesh.dim, cell_volume=mesh.cell_volume[cells], cell_centroid=mesh.cell_centroid[cells],
                       face_owner=new_own, face_neighbor=new_nei, face_area=mesh.face_area[keep], face_normal=nrm,
                       face_centroid=cen, face_shift=shift, bc=list(mesh.bc) + [BC(BC_OUTFLOW)],
                       name=mesh.name + "_patch")

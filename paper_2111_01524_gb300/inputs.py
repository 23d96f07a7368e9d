"""Seeded synthetic inputs: meshes and initial volume fractions.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds none of the advection or reconstruction arithmetic: it builds face-based
polyhedral meshes (the OpenFOAM-like layout of Sec. 3.1: planar polygonal
faces, owner/neighbour per face, face nodes counter-clockwise seen from
outside the owner) and fills the initial volume fraction field by adaptive
tetrahedral refinement against an implicit body (the role of ``initfgrid``,
Sec. 3.2), which is test-problem set-up, not part of the time step.

Mesh families (Sec. 4, grid list):
  * ``hex_mesh``     -- uniform grid of rectangular-parallelepiped cells.
  * ``kuhn_tet_mesh``-- each cube split into 6 tetrahedra along its main
                        diagonal, interior vertices jittered (stands in for
                        the TetGen grids, which are not available here).
  * ``trihex_mesh``  -- distorted cubic cells whose faces are triangulated
                        through the face centre: 14 vertices, 24 triangular
                        faces, generally non-convex (Sec. 4, third bullet).

Every mesh is returned as a dict of numpy arrays:
  X          float64 [n_vert, 3]  vertex coordinates
  face_ptr   int64   [n_face+1]   CSR offsets into face_vert
  face_vert  int32   [...]        face node loops
  owner      int32   [n_face]
  neighbour  int32   [n_face]     -1 on the domain boundary
  n_cell     int
  cell_tets  callable(cells) -> (tets [m, 4, 3], cell of each tet [m]): a
             tetrahedral decomposition of the given cells (``init_fraction``)
  cell_corners callable(cells) -> vertex ids of the cells' corners (or None)
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "hex_mesh", "kuhn_tet_mesh", "trihex_mesh", "Body", "sphere", "ellipsoid",
    "init_fraction", "mesh_counts", "Velocity", "deformation", "rotation",
    "translation",
]


# ----------------------------------------------------------------------------
# prescribed velocity fields (parameters only; each side evaluates them)
# ----------------------------------------------------------------------------
class Velocity:
    """Parameters of a prescribed velocity field of Sec. 4.2.

    kind 1: 3D deformation with period ``period`` (Sec. 4.2.3);
    kind 2: rigid rotation about the z-parallel axis through ``center`` with
            angular rate ``omega`` (Sec. 4.2.2);
    kind 3: uniform translation ``u0`` (Sec. 4.2.1);
    kind 4: 2D deformation in the x-z plane with period ``period`` (Sec. 4.3).
    """

    DEFORMATION, ROTATION, TRANSLATION, DEFORMATION2D = 1, 2, 3, 4

    def __init__(self, kind, period=3.0, omega=0.0, center=(0.5, 0.5, 0.5),
                 u0=(0.0, 0.0, 0.0)):
        self.kind = int(kind)
        self.period = float(period)
        self.omega = float(omega)
        self.center = tuple(float(c) for c in center)
        self.u0 = tuple(float(c) for c in u0)

    def __repr__(self):
        return (f"Velocity(kind={self.kind}, period={self.period}, omega={self.omega}, "
                f"center={self.center}, u0={self.u0})")


def deformation(period=3.0):
    return Velocity(Velocity.DEFORMATION, period=period)


def rotation(omega=2.0 * np.pi, center=(0.5, 0.5, 0.5)):
    return Velocity(Velocity.ROTATION, omega=omega, center=center)


def translation(u0):
    return Velocity(Velocity.TRANSLATION, u0=u0)


def deformation2d(period=8.0):
    return Velocity(Velocity.DEFORMATION2D, period=period)


# ----------------------------------------------------------------------------
# uniform / jittered hexahedral grids
# ----------------------------------------------------------------------------
def _grid_vertices(n, lo, hi, jitter, rng):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    h = (hi - lo) / n
    idx = np.arange(n + 1)
    k, j, i = np.meshgrid(idx, idx, idx, indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    X = lo + X * h
    if jitter > 0.0:
        I = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
        interior = np.all((I > 0) & (I < n), axis=1)
        d = rng.uniform(-jitter, jitter, size=(int(interior.sum()), 3)) * h
        X[interior] += d
    return X, h


def _vid(n, i, j, k):
    n1 = np.int64(n + 1)
    return i + n1 * (j + n1 * k)


def _cid(n, i, j, k):
    n0 = np.int64(n)
    return i + n0 * (j + n0 * k)


def _hex_faces(n):
    """Quad faces of an n^3 block: (loops[m,4], owner[m], neighbour[m]).

    Internal faces point from the lower-index cell (owner) to the upper one;
    boundary faces point out of the domain. Loops are counter-clockwise seen
    from outside the owner, i.e. their right-hand normal leaves the owner.
    """
    loops, own, nbr = [], [], []
    r = np.arange(n)
    rp = np.arange(n + 1)
    # x-faces: plane i = const, base loop normal +x
    k, j, i = np.meshgrid(r, r, rp, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    L = np.stack([_vid(n, i, j, k), _vid(n, i, j + 1, k),
                  _vid(n, i, j + 1, k + 1), _vid(n, i, j, k + 1)], axis=1)
    lower = np.where(i > 0, _cid(n, np.maximum(i - 1, 0), j, k), -1)
    upper = np.where(i < n, _cid(n, np.minimum(i, n - 1), j, k), -1)
    loops.append(L); own.append(lower); nbr.append(upper)
    # y-faces: base loop normal +y
    k, j, i = np.meshgrid(r, rp, r, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    L = np.stack([_vid(n, i, j, k), _vid(n, i, j, k + 1),
                  _vid(n, i + 1, j, k + 1), _vid(n, i + 1, j, k)], axis=1)
    lower = np.where(j > 0, _cid(n, i, np.maximum(j - 1, 0), k), -1)
    upper = np.where(j < n, _cid(n, i, np.minimum(j, n - 1), k), -1)
    loops.append(L); own.append(lower); nbr.append(upper)
    # z-faces: base loop normal +z
    k, j, i = np.meshgrid(rp, r, r, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    L = np.stack([_vid(n, i, j, k), _vid(n, i + 1, j, k),
                  _vid(n, i + 1, j + 1, k), _vid(n, i, j + 1, k)], axis=1)
    lower = np.where(k > 0, _cid(n, i, j, np.maximum(k - 1, 0)), -1)
    upper = np.where(k < n, _cid(n, i, j, np.minimum(k, n - 1)), -1)
    loops.append(L); own.append(lower); nbr.append(upper)

    L = np.concatenate(loops)
    lower = np.concatenate(own)
    upper = np.concatenate(nbr)
    owner = np.where(lower >= 0, lower, upper)
    neighbour = np.where(lower >= 0, upper, -1)
    # boundary faces whose only cell is the upper one point the other way
    flip = lower < 0
    L[flip] = L[flip][:, ::-1]
    return L.astype(np.int32), owner.astype(np.int32), neighbour.astype(np.int32)


def _hex_cell_corners(n):
    r = np.arange(n)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    c = {}
    for b in range(8):
        bi, bj, bk = b & 1, (b >> 1) & 1, (b >> 2) & 1
        c[(bi, bj, bk)] = _vid(n, i + bi, j + bj, k + bk)
    return c


# the 6 tetrahedra of a cube sharing the diagonal 000-111 (one per axis order)
_KUHN_PATHS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _kuhn_tets_of_cubes(corner):
    tets = []
    for p in _KUHN_PATHS:
        a = [0, 0, 0]
        verts = [corner[(0, 0, 0)]]
        for ax in p:
            a[ax] = 1
            verts.append(corner[tuple(a)])
        tets.append(np.stack(verts, axis=1))
    return tets  # list of [n_cube, 4] vertex ids


def _tet_volumes(P):
    a, b, c, d = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    return np.einsum("ij,ij->i", b - a, np.cross(c - a, d - a)) / 6.0


def _csr(loops):
    m, k = loops.shape
    ptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    return ptr, loops.reshape(-1).astype(np.int32)


def hex_mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), jitter=0.0, seed=0):
    """Uniform n^3 grid of rectangular-parallelepiped cells on [lo, hi].

    ``jitter`` > 0 moves interior vertices by U[-jitter*h, jitter*h] per
    component (faces then become non-planar; only used as the base of
    ``trihex_mesh``, which triangulates them).
    """
    rng = np.random.default_rng(seed)
    X, h = _grid_vertices(n, lo, hi, jitter, rng)
    L, owner, nbr = _hex_faces(n)
    ptr, fv = _csr(L)

    def corners(cells):
        cells = np.asarray(cells, np.int64)
        i, j, k = cells % n, (cells // n) % n, cells // (n * n)
        ids = [_vid(n, i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)) for b in range(8)]
        return np.stack(ids, axis=1)

    def tets(cells):
        c = corners(cells)
        T = []
        for p in _KUHN_PATHS:
            a = [0, 0, 0]
            v = [c[:, 0]]
            for ax in p:
                a[ax] = 1
                v.append(c[:, a[0] + 2 * a[1] + 4 * a[2]])
            T.append(np.stack(v, axis=1))
        T = np.stack(T, axis=1).reshape(-1, 4)
        return X[T], np.repeat(np.asarray(cells, np.int64), 6)

    box = None
    if jitter == 0.0:
        lo_ = np.asarray(lo, np.float64)

        def box(cells):
            cells = np.asarray(cells, np.int64)
            ijk = np.stack([cells % n, (cells // n) % n, cells // (n * n)], axis=1)
            return lo_ + ijk * h, h

    return dict(X=X, face_ptr=ptr, face_vert=fv, owner=owner, neighbour=nbr,
                n_cell=n ** 3, cell_corners=corners, cell_tets=tets, cell_box=box,
                kind="hex", n=n, h=h)


def slab_mesh(n):
    """Quasi-2D grid of the 2D tests (Sec. 4.3): n x 1 x n cells on the unit
    cube, one cell across y (the paper's 3D grids with a single cell along
    one coordinate direction, Sec. 3.2). Faces as in ``hex_mesh``: internal
    faces leave the lower-index cell, boundary faces leave the domain."""
    n1 = n + 1

    def vid(i, j, k):
        return i + n1 * (j + 2 * k)

    def cid(i, k):
        return i + n * k
    r, rp = np.arange(n), np.arange(n1)
    loops, lower, upper = [], [], []
    # x-faces (plane i), loop normal +x
    k, i = np.meshgrid(r, rp, indexing="ij")
    i, k = i.ravel(), k.ravel()
    loops.append(np.stack([vid(i, 0, k), vid(i, 1, k), vid(i, 1, k + 1), vid(i, 0, k + 1)], 1))
    lower.append(np.where(i > 0, cid(np.maximum(i - 1, 0), k), -1))
    upper.append(np.where(i < n, cid(np.minimum(i, n - 1), k), -1))
    # y-faces (j = 0, 1), loop normal +y
    for j in (0, 1):
        k, i = np.meshgrid(r, r, indexing="ij")
        i, k = i.ravel(), k.ravel()
        loops.append(np.stack([vid(i, j, k), vid(i, j, k + 1), vid(i + 1, j, k + 1), vid(i + 1, j, k)], 1))
        lower.append(cid(i, k) if j == 1 else np.full(i.shape, -1))
        upper.append(cid(i, k) if j == 0 else np.full(i.shape, -1))
    # z-faces (plane k), loop normal +z
    k, i = np.meshgrid(rp, r, indexing="ij")
    i, k = i.ravel(), k.ravel()
    loops.append(np.stack([vid(i, 0, k), vid(i + 1, 0, k), vid(i + 1, 1, k), vid(i, 1, k)], 1))
    lower.append(np.where(k > 0, cid(i, np.maximum(k - 1, 0)), -1))
    upper.append(np.where(k < n, cid(i, np.minimum(k, n - 1)), -1))
    L = np.concatenate(loops)
    lo_, up_ = np.concatenate(lower), np.concatenate(upper)
    owner = np.where(lo_ >= 0, lo_, up_)
    neighbour = np.where(lo_ >= 0, up_, -1)
    flip = lo_ < 0
    L[flip] = L[flip][:, ::-1]
    kk, jj, ii = np.meshgrid(rp, np.arange(2), rp, indexing="ij")
    X = np.stack([ii.ravel() / n, jj.ravel().astype(np.float64), kk.ravel() / n], 1)
    ptr, fv = _csr(L.astype(np.int32))

    def corners(cells):
        cells = np.asarray(cells, np.int64)
        i, k = cells % n, cells // n
        return np.stack([vid(i + (b & 1), (b >> 1) & 1, k + ((b >> 2) & 1)) for b in range(8)], 1)

    return dict(X=X, face_ptr=ptr, face_vert=fv, owner=owner.astype(np.int32),
                neighbour=neighbour.astype(np.int32), n_cell=n * n, cell_corners=corners,
                kind="slab", n=n)


def kuhn_tet_mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), jitter=0.2, seed=0):
    """n^3 cubes, each split into 6 Kuhn tetrahedra (6 n^3 cells).

    Interior vertices are jittered by U[-jitter*h, jitter*h]^3; the seed is
    advanced until every tetrahedron keeps a positive volume.
    """
    corner = _hex_cell_corners(n)
    T = np.concatenate(_kuhn_tets_of_cubes(corner))  # [6 n^3, 4]
    X0, h = _grid_vertices(n, lo, hi, 0.0, None)
    # orient every tetrahedron positively on the undistorted grid
    neg = _tet_volumes(X0[T]) < 0
    T[neg] = T[neg][:, [0, 2, 1, 3]]
    for attempt in range(64):
        rng = np.random.default_rng(seed + 7919 * attempt)
        X, h = _grid_vertices(n, lo, hi, jitter, rng)
        vol = _tet_volumes(X[T])
        if np.all(vol > 1e-3 * np.prod(h) / 6.0):
            break
    else:  # pragma: no cover - jitter of 0.2h never inverts a Kuhn tet
        raise RuntimeError("could not generate a valid jittered tet mesh")
    nt = T.shape[0]
    # the 4 faces of each tet, opposite to vertex 0..3, oriented outward
    fl = np.stack([T[:, [1, 2, 3]], T[:, [0, 3, 2]], T[:, [0, 1, 3]], T[:, [0, 2, 1]]], axis=1)
    fl = fl.reshape(-1, 3)
    ftet = np.repeat(np.arange(nt, dtype=np.int64), 4)
    key = np.sort(fl, axis=1)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    ks = key[order]
    same_as_next = np.all(ks[1:] == ks[:-1], axis=1)
    first = np.ones(len(ks), bool)
    first[1:] = ~same_as_next
    starts = np.nonzero(first)[0]
    counts = np.diff(np.append(starts, len(ks)))
    o = order[starts]
    owner = ftet[o]
    loops = fl[o]
    neighbour = np.full(len(starts), -1, np.int64)
    pair = counts == 2
    neighbour[pair] = ftet[order[starts[pair] + 1]]
    # owner = lower cell index; the loop must be outward from the owner
    swap = pair & (neighbour < owner)
    o2 = order[starts[swap] + 1]
    owner_s, nbr_s = owner.copy(), neighbour.copy()
    owner_s[swap], nbr_s[swap] = neighbour[swap], owner[swap]
    loops[swap] = fl[o2]
    ptr, fv = _csr(loops)

    def corners(cells):
        return T[np.asarray(cells, np.int64)]

    def tets(cells):
        cells = np.asarray(cells, np.int64)
        return X[T[cells]], cells

    return dict(X=X, face_ptr=ptr, face_vert=fv, owner=owner_s.astype(np.int32),
                neighbour=nbr_s.astype(np.int32), n_cell=nt, cell_corners=corners,
                cell_tets=tets, kind="tet", n=n, h=h)


def trihex_mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), jitter=0.3, seed=0):
    """Distorted cubic grid with face-centre triangulated faces.

    Interior grid vertices are jittered by U[-jitter*h, jitter*h]^3; each
    (generally non-planar) quad face gets a centre vertex (the average of its
    4 corners) and is replaced by 4 triangles, so every cell has 14 vertices
    and 24 planar triangular faces and is in general non-convex.
    """
    for attempt in range(64):
        rng = np.random.default_rng(seed + 7919 * attempt)
        X, h = _grid_vertices(n, lo, hi, jitter, rng)
        L, owner, nbr = _hex_faces(n)
        nq = L.shape[0]
        nv0 = X.shape[0]
        C = X[L].mean(axis=1)
        Xall = np.concatenate([X, C])
        cid = (nv0 + np.arange(nq)).astype(np.int32)
        tri = np.stack([np.stack([cid, L[:, q], L[:, (q + 1) % 4]], axis=1) for q in range(4)],
                       axis=1).reshape(-1, 3)
        t_owner = np.repeat(owner, 4)
        t_nbr = np.repeat(nbr, 4)
        # decomposition of each cell into 24 tetrahedra from its vertex average
        nc = n ** 3
        cen = np.zeros((nc, 3))
        corner = _hex_cell_corners(n)
        for v in corner.values():
            cen += X[v]
        cen /= 8.0
        # every triangle gives one tet per adjacent cell, oriented outward
        P_o = np.concatenate([cen[t_owner][:, None, :], Xall[tri]], axis=1)
        inner = t_nbr >= 0
        tri_n = tri[inner][:, [0, 2, 1]]
        P_n = np.concatenate([cen[t_nbr[inner]][:, None, :], Xall[tri_n]], axis=1)
        P = np.concatenate([P_o, P_n])
        vol = _tet_volumes(P)
        # (centre, a, b, c) with (a, b, c) counter-clockwise seen from
        # outside is positively oriented when the cell is star-shaped
        # about its vertex average; require that for every tetrahedron
        if np.all(vol > 0):
            break
    else:  # pragma: no cover
        raise RuntimeError("could not generate a valid distorted grid")
    cot = np.concatenate([t_owner, t_nbr[inner]]).astype(np.int64)
    order = np.argsort(cot, kind="stable")
    P, cot = P[order], cot[order]
    start = np.searchsorted(cot, np.arange(nc + 1))
    ptr, fv = _csr(tri.astype(np.int32))

    def tets(cells):
        # every cell has 24 tetrahedra, stored contiguously after the sort
        cells = np.asarray(cells, np.int64)
        if len(cells) == 0:
            return P[:0], cot[:0]
        idx = (start[cells][:, None] + np.arange(24)[None, :]).reshape(-1)
        return P[idx], cot[idx]

    def corners(cells):
        # the 8 grid corners of the cell; its face centres are averages of
        # them, so the corners' bounding ball contains the whole cell
        cells = np.asarray(cells, np.int64)
        i, j, k = cells % n, (cells // n) % n, cells // (n * n)
        ids = [_vid(n, i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)) for b in range(8)]
        return np.stack(ids, axis=1)

    return dict(X=Xall, face_ptr=ptr, face_vert=fv, owner=t_owner.astype(np.int32),
                neighbour=t_nbr.astype(np.int32), n_cell=nc, cell_corners=corners,
                cell_tets=tets, kind="trihex", n=n, h=h)


def mesh_counts(mesh):
    return dict(n_vert=int(mesh["X"].shape[0]), n_face=int(mesh["owner"].shape[0]),
                n_cell=int(mesh["n_cell"]))


# ----------------------------------------------------------------------------
# implicit bodies and initial volume fraction
# ----------------------------------------------------------------------------
class Body:
    """Axis-aligned ellipsoid (a sphere when all semi-axes are equal).

    ``dist`` is a conservative signed distance: negative inside, and
    |dist(x)| never exceeds the true distance to the surface (it is exact for
    a sphere), so a ball of radius r around x with |dist(x)| > r lies wholly
    on one side.
    """

    def __init__(self, center, axes):
        self.center = np.asarray(center, np.float64)
        self.axes = np.asarray(axes, np.float64)

    def dist(self, P):
        q = (P - self.center) / self.axes
        rho = np.sqrt(np.einsum("...i,...i->...", q, q))
        return (rho - 1.0) * self.axes.min()

    def volume(self):
        return 4.0 / 3.0 * np.pi * float(np.prod(self.axes))


def sphere(center, radius):
    return Body(center, [radius, radius, radius])


class Shape:
    """Parameters of an initial fluid body for the refinement initialisation
    (``initfgrid``, Sec. 3.2): a description only, evaluated by the oracle
    and by the device routine on their own. kind 1: sphere (centre c, radius
    r); 2: infinite cylinder (axis through c along the unit vector a, radius
    r); 3: half-space a.(x - c) < 0 (a unit)."""
    SPHERE, CYLINDER, HALFSPACE = 1, 2, 3

    def __init__(self, kind, c, a=(0.0, 0.0, 1.0), r=0.0):
        self.kind = int(kind)
        self.c = tuple(float(v) for v in c)
        a = np.asarray(a, np.float64)
        self.a = tuple(float(v) for v in a / np.linalg.norm(a))
        self.r = float(r)


def shape_sphere(center, radius):
    return Shape(Shape.SPHERE, center, r=radius)


def shape_cylinder(point, axis, radius):
    return Shape(Shape.CYLINDER, point, axis, radius)


def shape_halfspace(point, normal):
    return Shape(Shape.HALFSPACE, point, normal)


def ellipsoid(center, axes):
    return Body(center, axes)


def _subdivide_tets(P):
    """Split each tetrahedron into 8 by its edge midpoints."""
    a, b, c, d = P[:, 0], P[:, 1], P[:, 2], P[:, 3]
    ab, ac, ad = (a + b) / 2, (a + c) / 2, (a + d) / 2
    bc, bd, cd = (b + c) / 2, (b + d) / 2, (c + d) / 2
    kids = [
        (a, ab, ac, ad), (ab, b, bc, bd), (ac, bc, c, cd), (ad, bd, cd, d),
        (ab, ac, ad, bd), (ab, ac, bc, bd), (ac, ad, bd, cd), (ac, bc, bd, cd),
    ]
    return np.concatenate([np.stack(k, axis=1) for k in kids])


def init_fraction(mesh, body, levels=4, chunk=1 << 18):
    """Initial F per cell: adaptive refinement of the cells' tetrahedra.

    Cells whose bounding ball lies on one side of the body are 0 or 1; the
    others are split into tetrahedra, and a tetrahedron whose ball (about its
    centroid) lies on one side is counted whole while the rest are split
    8-fold, up to ``levels`` times; leaves are classified by their centroid.
    Returns F (float64 [n_cell]) with values in [0, 1].
    """
    nc = int(mesh["n_cell"])
    X = mesh["X"]
    F = np.zeros(nc)
    band = []
    for s in range(0, nc, chunk):
        cells = np.arange(s, min(nc, s + chunk))
        if mesh.get("cell_corners") is not None:
            P = X[mesh["cell_corners"](cells)]
        else:
            P = mesh["cell_points"](cells)
        cen = P.mean(axis=1)
        r = np.sqrt(np.max(np.sum((P - cen[:, None, :]) ** 2, axis=2), axis=1))
        d = body.dist(cen)
        F[cells[d < -r]] = 1.0
        band.append(cells[np.abs(d) <= r])
    band = np.concatenate(band) if band else np.zeros(0, np.int64)
    if mesh.get("cell_box") is not None:
        # axis-aligned boxes: octree refinement with exact box volumes
        step = max(1, chunk // 16)
        for s in range(0, len(band), step):
            cells = band[s:s + step]
            lo, h = mesh["cell_box"](cells)
            m = len(cells)
            own = np.arange(m)
            size = np.asarray(h, np.float64).copy()
            inside = np.zeros(m)
            for level in range(levels + 1):
                if lo.shape[0] == 0:
                    break
                cen = lo + 0.5 * size
                r = 0.5 * float(np.linalg.norm(size))
                d = body.dist(cen)
                v = float(np.prod(size))
                full = d < -r
                inside += np.bincount(own[full], minlength=m) * v
                cut = ~(full | (d > r))
                if level == levels:
                    inside += np.bincount(own[cut & (d < 0.0)], minlength=m) * v
                    break
                lo, own = lo[cut], own[cut]
                size = 0.5 * size
                offs = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)],
                                np.float64) * size
                lo = (lo[:, None, :] + offs[None, :, :]).reshape(-1, 3)
                own = np.repeat(own, 8)
            F[cells] = inside / float(np.prod(h))
        return np.clip(F, 0.0, 1.0)
    step = max(1, chunk // 64)
    for s in range(0, len(band), step):
        cells = band[s:s + step]
        T, owner = mesh["cell_tets"](cells)
        local = np.searchsorted(cells, owner)
        m = len(cells)
        vol_cell = np.bincount(local, weights=np.abs(_tet_volumes(T)), minlength=m)
        inside = np.zeros(m)
        P, own = T, local
        for level in range(levels + 1):
            if P.shape[0] == 0:
                break
            cen = P.mean(axis=1)
            r = np.sqrt(np.max(np.sum((P - cen[:, None, :]) ** 2, axis=2), axis=1))
            d = body.dist(cen)
            v = np.abs(_tet_volumes(P))
            full = d < -r
            inside += np.bincount(own[full], weights=v[full], minlength=m)
            cut = ~(full | (d > r))
            if level == levels:
                leaf_in = cut & (d < 0.0)
                inside += np.bincount(own[leaf_in], weights=v[leaf_in], minlength=m)
                break
            P = _subdivide_tets(P[cut])
            own = np.tile(own[cut], 8)
        F[cells] = inside / vol_cell
    return np.clip(F, 0.0, 1.0)

"""Domain decomposition of one grid into parts with a halo of node rings.

A part is a sub-mesh of its own: the cells it owns plus every cell within
``rings`` node-neighbour rings of them (cells that share a node, the
neighbourhood of the method's stencils), all the faces of those cells, and
the nodes of those faces. Cells, faces and nodes keep the grid's order (a
part numbers them by increasing grid index), so every per-cell list the
library builds (faces of a cell, node neighbours, cells around a node) has
the grid's order, and every sum over such a list adds the same terms in the
same order. A face whose owner is outside the part keeps its neighbour as
owner, with its nodes reversed (its normal then points out of that cell);
such faces lie on the part's outer boundary only.

How deep the halo must be follows from what one step reads (Secs. 2.1, 2.2,
3.5). The new F of a cell needs V_F of its faces; a face's V_F needs the
PLIC planes and tags of the candidate cells, the node neighbours of its two
cells (two rings); a cell's plane needs F at its node neighbours (one more
ring). So after the halo cells receive F from their owners, three rings give
every owned cell the grid's result bit for bit. LSFIR's outer iteration
(Sec. 2.1.2) reads the neighbours' normals once per iteration: one ring per
iteration. The mixed path's reconciliation of FP32 noise moves a cell's
excess to its face neighbours and reads their room, which is their own new
F: two rings per round, three rounds.

The partition itself is a pure function of the grid and the part count
(slabs of equal cell count along the longest axis, or recursive coordinate
bisection), so every rank computes the same one without communicating.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PREC_FP64, PREC_MIXED = 0, 1
RECON_LSGIR, RECON_LSFIR = 0, 1
RECONCILE_ROUNDS = 3


def halo_rings(precision=PREC_FP64, recon=RECON_LSGIR, lsfir_iters=4):
    """Node rings a part's halo needs for a bit-identical step."""
    r = 3
    if recon == RECON_LSFIR:
        r += int(lsfir_iters)
    if precision == PREC_MIXED:
        r += 2 * RECONCILE_ROUNDS
    return r


def _arrays(mesh):
    fp = np.ascontiguousarray(mesh["face_ptr"], np.int64)
    fv = np.ascontiguousarray(mesh["face_vert"], np.int64)
    own = np.ascontiguousarray(mesh["owner"], np.int64)
    nbr = np.ascontiguousarray(mesh["neighbour"], np.int64)
    return fp, fv, own, nbr


def cell_centres(mesh):
    """Mean over a cell's faces of the face's node mean: a point inside every
    convex cell, used only to order cells for the partition."""
    fp, fv, own, nbr = _arrays(mesh)
    X = np.asarray(mesh["X"], np.float64)
    nc = int(mesh["n_cell"])
    lens = np.diff(fp)
    fc = np.add.reduceat(X[fv], fp[:-1], axis=0) / lens[:, None]
    cnt = np.bincount(own, minlength=nc).astype(np.float64)
    m = nbr >= 0
    cnt += np.bincount(nbr[m], minlength=nc)
    cc = np.empty((nc, 3))
    for d in range(3):
        s = np.bincount(own, weights=fc[:, d], minlength=nc)
        s += np.bincount(nbr[m], weights=fc[m, d], minlength=nc)
        cc[:, d] = s / cnt
    return cc


def slab_partition(mesh, n_parts, axis=None):
    """Part of each cell: slabs of equal cell count (to one cell) along
    ``axis`` (default: the longest extent of the grid), ties by cell index."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    nc = int(mesh["n_cell"])
    if n_parts > nc:
        raise ValueError("more parts than cells")
    cc = cell_centres(mesh)
    if axis is None:
        axis = int(np.argmax(cc.max(axis=0) - cc.min(axis=0)))
    order = np.lexsort((np.arange(nc), cc[:, axis]))
    part = np.empty(nc, np.int32)
    bounds = (np.arange(n_parts + 1) * nc) // n_parts
    for p in range(n_parts):
        part[order[bounds[p]:bounds[p + 1]]] = p
    return part


def rcb_partition(mesh, n_parts):
    """Recursive coordinate bisection: split the cells along the longest
    extent of their centres, in proportion to the parts on each side."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    nc = int(mesh["n_cell"])
    if n_parts > nc:
        raise ValueError("more parts than cells")
    cc = cell_centres(mesh)
    part = np.empty(nc, np.int32)

    def split(cells, p0, n):
        if n == 1:
            part[cells] = p0
            return
        pts = cc[cells]
        ax = int(np.argmax(pts.max(axis=0) - pts.min(axis=0)))
        order = cells[np.lexsort((cells, pts[:, ax]))]
        nl = n // 2
        cut = (cells.size * nl) // n
        split(order[:cut], p0, nl)
        split(order[cut:], p0 + nl, n - nl)

    split(np.arange(nc), 0, n_parts)
    return part


def grow_rings(mesh, seed, rings):
    """Ring number of every cell from the seed cells (0), through cells that
    share a node with the previous ring, up to ``rings``; -1 beyond."""
    fp, fv, own, nbr = _arrays(mesh)
    nc = int(mesh["n_cell"])
    nv = int(np.asarray(mesh["X"]).shape[0])
    lens = np.diff(fp)
    fid = np.repeat(np.arange(own.size), lens)
    ring = np.full(nc, -1, np.int32)
    ring[np.asarray(seed, bool)] = 0
    front = ring == 0
    has_nbr = nbr >= 0
    nbr_safe = np.where(has_nbr, nbr, 0)
    for r in range(1, rings + 1):
        # nodes of the front's cells: the nodes of faces with a front cell
        fmask = front[own] | (has_nbr & front[nbr_safe])
        nodes = np.zeros(nv, bool)
        nodes[fv[fmask[fid]]] = True
        # cells with a face on one of those nodes
        touch = np.maximum.reduceat(nodes[fv].astype(np.uint8), fp[:-1]).astype(bool)
        new = np.zeros(nc, bool)
        new[own[touch]] = True
        new[nbr[touch & has_nbr]] = True
        new &= ring < 0
        ring[new] = r
        front = new
        if not new.any():
            break
    return ring


@dataclass
class Subdomain:
    """Part ``part`` of a grid: a sub-mesh of its cells and halo, with the
    index lists of the halo exchange (local cell indices).

    cells: grid index of each local cell (increasing); ring: 0 for an owned
    cell, k for a halo cell k rings out; faces, nodes: grid indices of the
    local faces and nodes (increasing); mesh: the sub-mesh in the library's
    mesh form; recv[q]: the halo cells owned by part q, in increasing grid
    order; send[q]: the owned cells that are in part q's halo, in the order
    of q's recv[self.part]."""

    part: int
    cells: np.ndarray
    ring: np.ndarray
    faces: np.ndarray
    nodes: np.ndarray
    mesh: dict
    recv: dict = field(default_factory=dict)
    send: dict = field(default_factory=dict)

    @property
    def owned(self):
        return np.flatnonzero(self.ring == 0).astype(np.int32)

    @property
    def neighbours(self):
        return sorted(set(self.recv) | set(self.send))


def submesh(mesh, local):
    """The sub-mesh of the cells in boolean mask ``local`` (see the module
    docstring for the numbering and the boundary faces); returns the mesh
    dict and the grid indices of its cells, faces and nodes."""
    fp, fv, own, nbr = _arrays(mesh)
    X = np.asarray(mesh["X"], np.float64)
    nc = int(mesh["n_cell"])
    cells = np.flatnonzero(local)
    g2l = np.full(nc, -1, np.int64)
    g2l[cells] = np.arange(cells.size)
    has_nbr = nbr >= 0
    nbr_safe = np.where(has_nbr, nbr, 0)
    fmask = local[own] | (has_nbr & local[nbr_safe])
    faces = np.flatnonzero(fmask)
    o = g2l[own[faces]]
    n = np.where(has_nbr[faces], g2l[nbr_safe[faces]], -1)
    flip = o < 0
    o = np.where(flip, n, o)
    n = np.where(flip, -1, n)
    starts = fp[faces]
    lens = fp[faces + 1] - starts
    ptr = np.zeros(faces.size + 1, np.int64)
    np.cumsum(lens, out=ptr[1:])
    j = np.arange(ptr[-1]) - np.repeat(ptr[:-1], lens)
    rev = np.repeat(flip, lens)
    src = np.repeat(starts, lens) + np.where(rev, np.repeat(lens, lens) - 1 - j, j)
    fvg = fv[src]
    nodes = np.unique(fvg)
    sub = dict(X=np.ascontiguousarray(X[nodes]), face_ptr=ptr,
               face_vert=np.searchsorted(nodes, fvg).astype(np.int32),
               owner=o.astype(np.int32), neighbour=n.astype(np.int32), n_cell=int(cells.size))
    return sub, cells, faces, nodes


def decompose(mesh, part, rings):
    """Subdomains of every part of ``part`` (one int per cell), each with a
    halo of ``rings`` node rings and the exchange lists between them."""
    part = np.asarray(part, np.int32)
    nc = int(mesh["n_cell"])
    if part.shape != (nc,):
        raise ValueError("part must hold one entry per cell")
    if rings < 1:
        raise ValueError("rings must be >= 1")
    n_parts = int(part.max()) + 1
    subs = []
    for p in range(n_parts):
        ring = grow_rings(mesh, part == p, rings)
        sub, cells, faces, nodes = submesh(mesh, ring >= 0)
        subs.append(Subdomain(p, cells.astype(np.int64), ring[cells], faces, nodes, sub))
    for sd in subs:
        halo = np.flatnonzero(sd.ring > 0)
        owner = part[sd.cells[halo]]
        for q in np.unique(owner):
            q = int(q)
            mine = halo[owner == q]
            sd.recv[q] = mine.astype(np.int32)
            other = subs[q]
            loc = np.searchsorted(other.cells, sd.cells[mine])
            if not np.array_equal(other.cells[loc], sd.cells[mine]) or np.any(other.ring[loc] != 0):
                raise AssertionError("halo cell not owned by its part")
            other.send[sd.part] = loc.astype(np.int32)
    return subs


def assemble(subs, values, n_cell):
    """Grid array of per-cell values from each part's owned cells
    (``values[p]``: one value per local cell of part p)."""
    out = np.empty(n_cell, np.asarray(values[0]).dtype)
    for sd, v in zip(subs, values):
        o = sd.owned
        out[sd.cells[o]] = np.asarray(v)[o]
    return out

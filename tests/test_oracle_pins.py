"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
a closed form, a brute-force count, a Monte-Carlo integral with an error
bound, an invariant, or a number printed in the paper (tests/golden/).
"""
import math
import os

import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def winding_number(P, tris):
    """Winding number of a closed triangulated surface at points P (exact,
    solid angles by the van Oosterom-Strackee formula)."""
    w = np.zeros(len(P))
    for a, b, c in tris:
        A, B, Cc = a - P, b - P, c - P
        la, lb, lc = (np.linalg.norm(X, axis=1) for X in (A, B, Cc))
        num = np.einsum("ij,ij->i", A, np.cross(B, Cc))
        den = (la * lb * lc + np.einsum("ij,ij->i", A, B) * lc
               + np.einsum("ij,ij->i", A, Cc) * lb + np.einsum("ij,ij->i", B, Cc) * la)
        w += 2.0 * np.arctan2(num, den)
    return w / (4.0 * np.pi)


def fan_tris(verts, faces):
    out = []
    for f in faces:
        for i in range(1, len(f) - 1):
            out.append((verts[f[0]], verts[f[i]], verts[f[i + 1]]))
    return out


def sz_fraction_below(m, a):
    """Closed-form volume of {y in [0,1]^3 : m.y < a}, m_i > 0 (the
    inclusion-exclusion form of the cuboid cut used by the analytic method
    cited in Sec. 2.1)."""
    m1, m2, m3 = m
    F3 = lambda x: max(x, 0.0) ** 3
    s = m1 + m2 + m3
    if a <= 0:
        return 0.0
    if a >= s:
        return 1.0
    v = (F3(a) - F3(a - m1) - F3(a - m2) - F3(a - m3) + F3(a - m1 - m2)
         + F3(a - m1 - m3) + F3(a - m2 - m3) - F3(a - s))
    return v / (6.0 * m1 * m2 * m3)


def box_cut_fraction(n, C, h):
    """Fluid fraction of a box cell (edge h, centroid xc) for the plane
    n.(x - xc) + C >= 0, from the closed form."""
    K = 0.5 * sum(n) - C / h
    shift = sum(x for x in n if x < 0)
    m = [abs(x) for x in n]
    return 1.0 - sz_fraction_below(m, K - shift)


@pytest.fixture(scope="module")
def hex4(orc):
    m = I.hex_mesh(4)
    return m, orc.Mesh(m)


# ---------------------------------------------------------------- geometry
def test_hex_geometry_closed_form(hex4):
    m, om = hex4
    g = om.geometry()
    h = 0.25
    assert np.allclose(g["cell_vol"], h ** 3, rtol=0, atol=1e-17)
    # centroid of cell (i,j,k) is ((i+.5)h, (j+.5)h, (k+.5)h)
    c = np.arange(64)
    ijk = np.stack([c % 4, (c // 4) % 4, c // 16], axis=1)
    assert np.allclose(g["cell_cen"], (ijk + 0.5) * h, atol=1e-16)
    assert np.allclose(g["face_area"], h * h, atol=1e-17)
    assert np.allclose(np.abs(g["face_nrm"]).max(axis=1), 1.0)
    assert g["cell_convex"].all()
    # face normal leaves the owner: (face centre - owner centroid) . n > 0
    own = m["owner"]
    d = g["face_cen"] - g["cell_cen"][own]
    assert (np.einsum("ij,ij->i", d, g["face_nrm"]) > 0).all()


@pytest.mark.parametrize("gen", ["tet", "trihex"])
def test_unstructured_geometry(orc, gen):
    m = I.kuhn_tet_mesh(3, seed=5) if gen == "tet" else I.trihex_mesh(3, seed=5)
    om = orc.Mesh(m)
    g = om.geometry()
    assert abs(g["cell_vol"].sum() - 1.0) < 1e-14
    assert (g["cell_vol"] > 0).all()
    if gen == "tet":
        # centroid of a tetrahedron = average of its 4 vertices (closed form)
        T, _ = m["cell_tets"](np.arange(om.n_cell))
        assert np.allclose(g["cell_cen"], T.mean(axis=1), atol=1e-15)
        assert g["cell_convex"].all()
    else:
        # distorted cells: centroid from the independent tet decomposition
        T, cot = m["cell_tets"](np.arange(om.n_cell))
        v = np.einsum("ij,ij->i", T[:, 1] - T[:, 0], np.cross(T[:, 2] - T[:, 0], T[:, 3] - T[:, 0])) / 6
        cen = np.zeros((om.n_cell, 3))
        np.add.at(cen, cot, v[:, None] * T.mean(axis=1))
        vol = np.bincount(cot, weights=v)
        assert np.allclose(g["cell_cen"], cen / vol[:, None], atol=1e-15)
        assert not g["cell_convex"].all()


def test_neigbcell_bruteforce_hex(hex4):
    m, om = hex4
    ptr, idx = om.neighbors()
    n = 4
    for c in range(n ** 3):
        i, j, k = c % n, (c // n) % n, c // (n * n)
        exp = sorted(ii + n * (jj + n * kk)
                     for ii in range(i - 1, i + 2) for jj in range(j - 1, j + 2)
                     for kk in range(k - 1, k + 2)
                     if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n and (ii, jj, kk) != (i, j, k))
        assert list(idx[ptr[c]:ptr[c + 1]]) == exp


def test_neigbcell_bruteforce_tets(orc):
    m = I.kuhn_tet_mesh(2, seed=1)
    om = orc.Mesh(m)
    ptr, idx = om.neighbors()
    # vertex sets of the cells from the face loops
    fv, fp = m["face_vert"], m["face_ptr"]
    vs = [set() for _ in range(m["n_cell"])]
    for f in range(len(m["owner"])):
        loop = set(fv[fp[f]:fp[f + 1]])
        vs[m["owner"][f]] |= loop
        if m["neighbour"][f] >= 0:
            vs[m["neighbour"][f]] |= loop
    for c in range(m["n_cell"]):
        exp = [k for k in range(m["n_cell"]) if k != c and vs[c] & vs[k]]
        assert list(idx[ptr[c]:ptr[c + 1]]) == exp


# ---------------------------------------------------------------- tags
def test_taggrid_hand_cases(hex4):
    m, om = hex4
    F = np.zeros(64)
    st = om.taggrid(F)
    assert (st["tag_c"] == -1).all() and (st["tag_v"] == -1).all() and (st["tag_f"] == -1).all()
    st = om.taggrid(np.ones(64))
    assert (st["tag_c"] == 1).all() and (st["tag_f"] == 1).all()
    # one interfacial cell: it and its 26 node neighbours' shared nodes are 0
    F = np.zeros(64)
    c = 1 + 4 * (1 + 4 * 1)
    F[c] = 0.5
    F[0] = 1e-13        # below eps: cut off to 0
    F[63] = 1 - 1e-13   # above 1-eps: cut off to 1
    st = om.taggrid(F)
    assert st["F"][0] == 0.0 and st["F"][63] == 1.0
    assert st["tag_c"][c] == 0 and (st["tag_c"] == 0).sum() == 1
    assert st["tag_c"][63] == 1
    # the 8 nodes of cell c are tagged 0; every face touching them is 0
    fv, fp = m["face_vert"], m["face_ptr"]
    nodes_c = set()
    for f in range(len(m["owner"])):
        if c in (m["owner"][f], m["neighbour"][f]):
            nodes_c |= set(fv[fp[f]:fp[f + 1]])
    zero_nodes = set(np.nonzero(st["tag_v"] == 0)[0])
    assert nodes_c <= zero_nodes
    for f in range(len(m["owner"])):
        touches = bool(set(fv[fp[f]:fp[f + 1]]) & zero_nodes)
        assert (st["tag_f"][f] == 0) == touches


# ---------------------------------------------------------------- cut volume
def test_cut_volume_matches_cuboid_closed_form(hex4):
    m, om = hex4
    rng = np.random.default_rng(3)
    h = 0.25
    cell = 21
    V = h ** 3
    for _ in range(200):
        # the closed form divides by m1 m2 m3: keep it well conditioned
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        while np.min(np.abs(n)) < 0.05:
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
        C = rng.uniform(-0.9, 0.9) * h
        got = om.cell_cut_volume(cell, n, C) / V
        exp = box_cut_fraction(n, C, h)
        assert abs(got - exp) < 1e-13, (n, C, got, exp)


def test_cut_volume_matches_tetrahedron_corner_closed_form(orc):
    """A plane that leaves one vertex v0 of a tetrahedron on one side cuts
    off the tetrahedron spanned by v0 and the three edge points, whose
    volume is t1 t2 t3 V with t_i = phi(v0) / (phi(v0) - phi(v_i)) the edge
    fractions (phi the plane's signed distance): the fluid part is that
    corner when v0 is the one fluid vertex, and V minus it when v0 is the
    one empty vertex. Jittered Kuhn tetrahedra, random planes through the
    cell near each vertex."""
    m = I.kuhn_tet_mesh(3, seed=5)
    om = orc.Mesh(m)
    g = om.geometry()
    fv, fp = m["face_vert"], m["face_ptr"]
    rng = np.random.default_rng(17)
    checked = 0
    for c in rng.choice(m["n_cell"], 12, replace=False):
        faces = np.nonzero((m["owner"] == c) | (m["neighbour"] == c))[0]
        verts = np.unique(np.concatenate([fv[fp[f]:fp[f + 1]] for f in faces]))
        assert verts.size == 4
        X = m["X"][verts]
        V = abs(np.linalg.det(X[1:] - X[0])) / 6.0
        assert abs(V - g["cell_vol"][c]) < 1e-15
        xc = g["cell_cen"][c]
        for i0 in range(4):
            others = [i for i in range(4) if i != i0]
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            d = (X - xc) @ n
            if any(abs(d[i0] - d[i]) < 0.2 * np.ptp(d) for i in others):
                continue  # keep the edge fractions well conditioned
            side = 1.0 if all(d[i0] > d[i] for i in others) else (
                -1.0 if all(d[i0] < d[i] for i in others) else 0.0)
            if side == 0.0:
                continue
            # a plane strictly between v0 and the other three
            lim = max(d[i] for i in others) if side > 0 else min(d[i] for i in others)
            s = rng.uniform(0.2, 0.8)
            cut = lim + s * (d[i0] - lim)
            C = -cut                                  # n.(x - xc) + C = 0 at the cut
            t = [(d[i0] - cut) / (d[i0] - d[i]) for i in others]
            corner = t[0] * t[1] * t[2] * V
            exp = corner if side > 0 else V - corner  # fluid side: n.(x - xc) + C >= 0
            got = om.cell_cut_volume(int(c), n, C)
            assert abs(got - exp) < 1e-14 * V + 1e-18, (c, i0, got, exp)
            checked += 1
    assert checked >= 12


def test_cut_volume_monte_carlo_nonconvex(orc):
    m = I.trihex_mesh(2, seed=11)
    om = orc.Mesh(m)
    g = om.geometry()
    # pick a non-convex cell
    c = int(np.nonzero(g["cell_convex"] == 0)[0][0])
    fv, fp = m["face_vert"], m["face_ptr"]
    tris = []
    for f in range(len(m["owner"])):
        loop = list(fv[fp[f]:fp[f + 1]])
        if m["owner"][f] == c:
            tris.append(tuple(m["X"][v] for v in loop))
        elif m["neighbour"][f] == c:
            tris.append(tuple(m["X"][v] for v in loop[::-1]))
    bb = g["cell_bbox"][c]
    rng = np.random.default_rng(0)
    N = 400_000
    P = bb[:3] + rng.random((N, 3)) * (bb[3:] - bb[:3])
    w = winding_number(P, tris)
    box = np.prod(bb[3:] - bb[:3])
    assert abs(w.mean() * box - g["cell_vol"][c]) < 4 * box * np.sqrt(0.25 / N)
    n = np.array([0.3, -0.5, 0.8]); n /= np.linalg.norm(n)
    xc = g["cell_cen"][c]
    for C in (-0.2 * 0.5, 0.0, 0.13 * 0.5):
        inside = (w > 0.5) & ((P - xc) @ n + C >= 0)
        mc = inside.mean() * box
        got = om.cell_cut_volume(c, n, C)
        sig = box * np.sqrt(inside.mean() * (1 - inside.mean()) / N)
        assert abs(got - mc) < 4 * sig + 1e-12, (C, got, mc)


def test_plane_constant_solves_volume_equation(hex4):
    m, om = hex4
    rng = np.random.default_rng(7)
    F = rng.uniform(0.0, 1.0, size=64)
    F[:5] = [1e-11, 1 - 1e-11, 0.5, 1e-6, 1 - 1e-6]
    st = om.taggrid(F)
    nrm = rng.normal(size=(64, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    Cc = om.plane_constant(st["F"], st["tag_c"], nrm)
    h = 0.25
    for c in range(64):
        if st["tag_c"][c] != 0:
            continue
        # closed form of the cuboid cut volume at the found C
        got = box_cut_fraction(nrm[c], Cc[c], h)
        assert abs(got - st["F"][c]) < 1e-13


def test_plane_constant_symmetric_half(orc):
    # F = 0.5 in a centrally symmetric cell: the plane passes through the
    # centroid (C = 0) for any normal
    m = I.hex_mesh(2)
    om = orc.Mesh(m)
    F = np.full(8, 0.5)
    st = om.taggrid(F)
    rng = np.random.default_rng(1)
    nrm = rng.normal(size=(8, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    Cc = om.plane_constant(st["F"], st["tag_c"], nrm)
    assert np.abs(Cc).max() < 1e-15


# ---------------------------------------------------------------- truncation
CUBE_V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                   [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
CUBE_F = [[0, 3, 2, 1], [4, 5, 6, 7], [0, 1, 5, 4], [2, 3, 7, 6], [1, 2, 6, 5], [0, 4, 7, 3]]


def test_clip_box_by_box_closed_form(orc):
    rng = np.random.default_rng(2)
    assert abs(orc.poly_volume(CUBE_V, CUBE_F) - 1.0) < 1e-15
    for _ in range(50):
        lo = rng.uniform(-0.5, 1.0, 3)
        hi = lo + rng.uniform(0.1, 1.0, 3)
        planes = []
        for d in range(3):
            a = np.zeros(3); a[d] = 1.0
            planes.append(list(a) + [-lo[d]])
            planes.append(list(-a) + [hi[d]])
        exp = np.prod(np.clip(np.minimum(hi, 1) - np.maximum(lo, 0), 0, None))
        got = orc.poly_clip_volume(CUBE_V, CUBE_F, planes)
        assert abs(got - exp) < 1e-14


def test_clip_self_intersecting_monte_carlo(orc):
    # a "bow-tie" prism: top face twisted by 180 degrees -> self-intersecting
    # side faces; signed volume is a winding-number integral
    rng = np.random.default_rng(4)
    bot = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], float)
    top = np.array([[1, 1, 1], [0, 1, 1], [0, 0, 1], [1, 0, 1]], float) + rng.normal(0, 0.05, (4, 3))
    V = np.concatenate([bot, top])
    faces = [[0, 3, 2, 1], [4, 5, 6, 7]] + [[i, (i + 1) % 4, 4 + (i + 1) % 4, 4 + i] for i in range(4)]
    # split the (non-planar) quads into triangles to have a proper surface
    tri_faces = []
    for f in faces:
        tri_faces += [[f[0], f[1], f[2]], [f[0], f[2], f[3]]]
    tris = fan_tris(V, tri_faces)
    N = 300_000
    lo, hi = V.min(0) - 0.01, V.max(0) + 0.01
    P = lo + rng.random((N, 3)) * (hi - lo)
    w = winding_number(P, tris)
    box = np.prod(hi - lo)
    plane = np.array([0.4, -0.3, 0.7]); plane /= np.linalg.norm(plane)
    for b in (-0.5, -0.2, 0.1):
        sel = (P @ plane + b) > 0
        mc = (w * sel).mean() * box
        sig = box * np.sqrt(np.var(w * sel) / N)
        got = orc.poly_clip_volume(V, tri_faces, [list(plane) + [b]])
        assert abs(got - mc) < 4 * sig + 1e-9, (b, got, mc)
    assert abs(orc.poly_volume(V, tri_faces) - w.mean() * box) < 4 * box * np.sqrt(np.var(w) / N)


# ---------------------------------------------------------------- FMFPA
def test_fmfpa_uniform_velocity_is_parallelepiped(orc):
    m = I.kuhn_tet_mesh(3, seed=2)
    om = orc.Mesh(m)
    u = (0.3, -0.2, 0.5)
    vel = I.translation(u)
    dt = 0.01
    g = om.geometry()
    for f in range(0, len(m["owner"]), 7):
        P, vd, fl = om.fmfpa(f, vel, 0.0, dt)
        nI = m["face_ptr"][f + 1] - m["face_ptr"][f]
        assert P.shape[0] == 2 * nI + 1  # 2I+1 vertices (Sec. 2.2.2)
        X = m["X"][m["face_vert"][m["face_ptr"][f]:m["face_ptr"][f + 1]]]
        assert np.allclose(P[nI:2 * nI], X - dt * np.array(u), atol=1e-15)
        # apex = centroid of the back-traced face (no volume correction)
        assert np.allclose(P[2 * nI], (X - dt * np.array(u)).mean(0), atol=1e-14)
        assert abs(vd - np.dot(u, g["face_nrm"][f]) * g["face_area"][f] * dt) < 1e-18


def _fmfpa_faces(nI):
    faces = [list(range(nI))]
    for i in range(nI):
        ip = (i + 1) % nI
        faces.append([ip, i, nI + i, nI + ip])
    for i in range(nI):
        ip = (i + 1) % nI
        faces.append([nI + ip, nI + i, 2 * nI])
    return faces


@pytest.mark.parametrize("gen", ["hex", "tet"])
def test_fmfpa_volume_equals_vd(orc, gen):
    m = I.hex_mesh(6) if gen == "hex" else I.kuhn_tet_mesh(4, seed=3)
    om = orc.Mesh(m)
    vel = I.deformation(3.0)
    dt = 0.5 / 6 / 2
    A = om.geometry()["face_area"]
    for f in range(0, len(m["owner"]), 3):
        P, vd, fl = om.fmfpa(f, vel, 0.2, dt)
        nI = (P.shape[0] - 1) // 2
        if fl & 2:
            continue
        vol = orc.poly_volume(P - P[:nI].mean(0), _fmfpa_faces(nI))
        # roundoff is relative to the face scale A^(3/2), not to V_d
        assert abs(vol - vd) <= 1e-14 * max(abs(vd), A[f] ** 1.5), (f, vol, vd)


def test_fmfpa_face_matching(orc):
    """Flux polyhedra of two faces sharing an edge have coplanar side faces
    on that edge (the face-matched property, Sec. 2.2.2)."""
    m = I.kuhn_tet_mesh(3, seed=9)
    om = orc.Mesh(m)
    vel = I.deformation(3.0)
    fv, fp = m["face_vert"], m["face_ptr"]
    edges = {}
    for f in range(len(m["owner"])):
        loop = list(fv[fp[f]:fp[f + 1]])
        for i in range(len(loop)):
            e = tuple(sorted((loop[i], loop[(i + 1) % len(loop)])))
            edges.setdefault(e, []).append((f, i))
    checked = 0
    for e, lst in edges.items():
        if len(lst) < 2:
            continue
        (f1, i1), (f2, i2) = lst[0], lst[1]
        P1, _, fl1 = om.fmfpa(f1, vel, 0.3, 0.02)
        P2, _, fl2 = om.fmfpa(f2, vel, 0.3, 0.02)
        if fl1 or fl2:
            continue
        n1 = (P1.shape[0] - 1) // 2
        n2 = (P2.shape[0] - 1) // 2
        # side plane on this edge: contains the edge, parallel to the
        # velocity at the edge centre
        a, b = P1[i1], P1[(i1 + 1) % n1]
        ue = om.velocity(vel, 0.5 * (a + b), 0.3)
        nrm = np.cross(b - a, ue)
        if np.linalg.norm(nrm) < 1e-6 * np.linalg.norm(b - a):
            continue
        nrm /= np.linalg.norm(nrm)
        # face 1's own back-traced points lie in it
        for k in (i1, (i1 + 1) % n1):
            assert abs(np.dot(P1[n1 + k] - a, nrm)) < 1e-15
        # the back-traced points of face 2 on the same edge lie in it
        j = [P2[k] for k in range(n2)]
        for k in (i2, (i2 + 1) % n2):
            assert abs(np.dot(P2[n2 + k] - a, nrm)) < 1e-15
        checked += 1
        if checked > 40:
            break
    assert checked > 10


# ---------------------------------------------------------------- EMFPA
def _emfpa_faces(nI):
    """Faces of the edge-matched polyhedron as Sec. 2.2.1 states them: the
    cell face; each side face (edge i, the two streak lines, the back-traced
    edge) as four triangles around its centre s_i; the back-traced loop as a
    fan of I triangles around the apex."""
    faces = [list(range(nI))]
    for i in range(nI):
        ip = (i + 1) % nI
        side = [ip, i, nI + i, nI + ip]
        faces += [[side[e], side[(e + 1) % 4], 2 * nI + i] for e in range(4)]
    faces += [[nI + (i + 1) % nI, nI + i, 3 * nI] for i in range(nI)]
    return faces


def _face_nodes(m, f):
    return m["X"][m["face_vert"][m["face_ptr"][f]:m["face_ptr"][f + 1]]]


def _rot_u(x, omega, c):
    """rigid rotation about the z-parallel axis through c, written out"""
    return np.stack([-omega * (x[:, 1] - c[1]), omega * (x[:, 0] - c[0]), 0.0 * x[:, 2]], 1)


def test_emfpa_uniform_velocity_is_prism(orc):
    m = I.kuhn_tet_mesh(3, seed=2)
    om = orc.Mesh(m)
    u = np.array((0.3, -0.2, 0.5))
    vel = I.translation(u)
    dt = 0.01
    g = om.geometry()
    for f in range(0, len(m["owner"]), 5):
        P, vd, fl = om.emfpa(f, vel, 0.0, dt)
        X = _face_nodes(m, f)
        nI = len(X)
        assert P.shape[0] == 3 * nI + 1  # 3I+1 vertices (Sec. 2.2.1)
        assert np.allclose(P[:nI], X, atol=1e-15)
        assert np.allclose(P[nI:2 * nI], X - dt * u, atol=1e-15)
        # a uniform field makes every side face a planar parallelogram and
        # the polyhedron the exact prism: the apex needs no correction
        assert np.allclose(P[3 * nI], (X - dt * u).mean(0), atol=1e-14)
        assert abs(vd - u @ g["face_nrm"][f] * g["face_area"][f] * dt) < 1e-18
        assert len(_emfpa_faces(nI)) == 5 * nI + 1


@pytest.mark.parametrize("gen", ["hex", "tet"])
def test_emfpa_rotation_backtrace_and_volume(orc, gen):
    """Rigid rotation: each vertex goes back along its own streak line with
    its own velocity (Eq. streak-line2), the side centres are vertex
    averages, and the apex lies on the normal through the centroid of the
    back-traced loop at the height that makes the volume V_d."""
    m = I.hex_mesh(5) if gen == "hex" else I.kuhn_tet_mesh(4, seed=5)
    om = orc.Mesh(m)
    g = om.geometry()
    omega, c = 2.0 * np.pi, (0.5, 0.5, 0.5)
    vel = I.rotation(omega, c)
    dt = 0.02
    n_checked = 0
    for f in range(0, len(m["owner"]), 3):
        P, vd, fl = om.emfpa(f, vel, 0.1, dt)
        X = _face_nodes(m, f)
        nI = len(X)
        xb = X - dt * _rot_u(X, omega, c)
        assert np.allclose(P[nI:2 * nI], xb, atol=1e-15)
        for i in range(nI):
            ip = (i + 1) % nI
            ctr = 0.25 * (X[i] + X[ip] + xb[i] + xb[ip])
            assert np.allclose(P[2 * nI + i], ctr, atol=1e-15)
        # apex on the normal line through the centroid of the back-traced loop
        d = P[3 * nI] - xb.mean(0)
        assert np.linalg.norm(np.cross(d, g["face_nrm"][f])) < 1e-14
        if fl & 2:
            continue
        o = X.mean(0)
        vol = orc.poly_volume(P - o, _emfpa_faces(nI))
        A = g["face_area"][f]
        assert abs(vol - vd) <= 1e-14 * max(abs(vd), A ** 1.5), (f, vol, vd)
        n_checked += 1
    assert n_checked > 20


def test_emfpa_backtrace_uses_midtime_velocity(orc):
    """The time-modulated deformation field (Sec. 4.2), written out: the
    back-traced vertex uses the velocity at t^{n+1/2} = t + dt/2."""
    m = I.trihex_mesh(2, seed=7)
    om = orc.Mesh(m)
    T, t, dt = 3.0, 0.4, 0.05
    vel = I.deformation(T)

    def u(x, tt):
        s, s2 = np.sin(np.pi * x), np.sin(2 * np.pi * x)
        gt = np.cos(np.pi * tt / T)
        return gt * np.stack([2 * s[:, 0] ** 2 * s2[:, 1] * s2[:, 2],
                              -s2[:, 0] * s[:, 1] ** 2 * s2[:, 2],
                              -s2[:, 0] * s2[:, 1] * s[:, 2] ** 2], 1)

    for f in range(0, len(m["owner"]), 4):
        P, _, _ = om.emfpa(f, vel, t + 0.5 * dt, dt)
        X = _face_nodes(m, f)
        nI = len(X)
        assert np.allclose(P[nI:2 * nI], X - dt * u(X, t + 0.5 * dt), atol=1e-15)
    # and the whole step hands faceflux t, not the mid-time
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.45, 0.5, 0.5), 0.3), levels=2))
    Vd, _, _ = om.faceflux(vel, t, dt, st, orc.EMFPA)
    g = om.geometry()
    uc = u(g["face_cen"], t + 0.5 * dt)
    assert np.allclose(Vd, (uc * g["face_nrm"]).sum(1) * g["face_area"] * dt, atol=1e-17)


@pytest.mark.parametrize("gen", ["hex", "tet", "trihex"])
def test_emfpa_volume_equals_vd(orc, gen):
    m = {"hex": lambda: I.hex_mesh(6),
         "tet": lambda: I.kuhn_tet_mesh(4, seed=3),
         "trihex": lambda: I.trihex_mesh(3, seed=2)}[gen]()
    om = orc.Mesh(m)
    vel = I.deformation(3.0)
    dt = 0.5 / 6 / 2
    A = om.geometry()["face_area"]
    n_checked = 0
    for f in range(0, len(m["owner"]), 3):
        P, vd, fl = om.emfpa(f, vel, 0.2, dt)
        nI = (P.shape[0] - 1) // 3
        if fl & 2:
            continue
        vol = orc.poly_volume(P - P[:nI].mean(0), _emfpa_faces(nI))
        assert abs(vol - vd) <= 1e-14 * max(abs(vd), A[f] ** 1.5), (f, vol, vd)
        n_checked += 1
    assert n_checked > 20


def test_emfpa_edge_matching(orc):
    """Polyhedra of two faces sharing an edge have the same four side
    triangles on it, and polyhedra of faces sharing a vertex the same
    back-traced point: no over/underlap along shared edges and streak lines
    (the edge-matched property, Sec. 2.2.1)."""
    m = I.kuhn_tet_mesh(3, seed=9)
    om = orc.Mesh(m)
    vel = I.deformation(3.0)
    fv, fp = m["face_vert"], m["face_ptr"]
    polys = {}

    def poly(f):
        if f not in polys:
            polys[f] = om.emfpa(f, vel, 0.3, 0.02)[0]
        return polys[f]

    edges, verts = {}, {}
    for f in range(len(m["owner"])):
        loop = list(fv[fp[f]:fp[f + 1]])
        for i in range(len(loop)):
            e = tuple(sorted((loop[i], loop[(i + 1) % len(loop)])))
            edges.setdefault(e, []).append((f, i))
            verts.setdefault(loop[i], []).append((f, i))
    checked = 0
    for e, lst in edges.items():
        if len(lst) < 2:
            continue
        sides = []
        for f, i in lst[:3]:
            P = poly(f)
            nI = (P.shape[0] - 1) // 3
            ip = (i + 1) % nI
            ends = {fv[fp[f] + i]: (P[i], P[nI + i]), fv[fp[f] + ip]: (P[ip], P[nI + ip])}
            sides.append((ends, P[2 * nI + i]))
        (e0, s0) = sides[0]
        for ends, sc in sides[1:]:
            assert np.allclose(sc, s0, atol=1e-15)
            for v in e:
                assert np.allclose(ends[v][0], e0[v][0], atol=1e-15)
                assert np.allclose(ends[v][1], e0[v][1], atol=1e-15)
        checked += 1
        if checked > 60:
            break
    assert checked > 20
    for v, lst in list(verts.items())[:40]:
        pts = []
        for f, i in lst:
            P = poly(f)
            nI = (P.shape[0] - 1) // 3
            pts.append(P[nI + i])
        assert np.ptp(np.array(pts), axis=0).max() < 1e-15


def test_emfpa_and_fmfpa_agree_for_uniform_flow(orc):
    """A uniform field gives both constructions the same exact prism on
    every face (planar sides, no apex correction), so their fluid volumes
    agree up to rounding although the surfaces are triangulated
    differently."""
    m = I.kuhn_tet_mesh(5, seed=8)
    om = orc.Mesh(m)
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.22), levels=3))
    vel = I.translation((0.4, -0.3, 0.2))
    dt = om.suggest_dt(vel, 0.0, 0.6, 10.0)
    Vd0, VF0, s0 = om.faceflux(vel, 0.0, dt, st, orc.FMFPA)
    Vd1, VF1, s1 = om.faceflux(vel, 0.0, dt, st, orc.EMFPA)
    assert np.array_equal(Vd0, Vd1)
    assert s0[0] == s1[0] > 50  # the same geometric faces
    assert np.abs(VF1 - VF0).max() < 1e-15 * np.abs(Vd0).max() * 100


def test_emfpa_cfl1_translation_shifts_exactly(orc):
    """u = (1,0,0), dt = h on a uniform grid: each x-face EMFPA polyhedron is
    the upstream cell and the others are flat, so F moves one cell per step
    for ANY F."""
    n = 6
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    F0 = I.init_fraction(m, I.sphere((0.45, 0.52, 0.48), 0.27), levels=3)
    st = om.reconstruct(F0)
    vel = I.translation((1.0, 0.0, 0.0))
    new = om.step(vel, 0.0, 1.0 / n, st, method=orc.EMFPA)
    F = st["F"].reshape(n, n, n)
    G = new["F_unclipped_cut"].reshape(n, n, n)
    assert np.abs(G[:, :, 1:] - F[:, :, :-1]).max() < 2e-15
    assert np.abs(G[:, :, 0]).max() == 0.0


def test_emfpa_deformation_conserves_volume(orc):
    m = I.hex_mesh(16)
    om = orc.Mesh(m)
    V = om.geometry()["cell_vol"]
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15)))
    vel = I.deformation(3.0)
    t = 0.0
    for _ in range(4):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        v0 = (V * st["F"]).sum()
        new = om.step(vel, t, dt, st, method=orc.EMFPA)
        assert abs((V * new["F_unclipped_cut"]).sum() - v0) < 1e-13 * v0
        st, t = new, t + dt


# ---------------------------------------------------------------- LSGIR
def test_lsgir_exact_for_linear_field(orc):
    m = I.kuhn_tet_mesh(4, seed=4)
    om = orc.Mesh(m)
    g = om.geometry()
    a = np.array([0.3, -0.5, 0.2])
    F = 0.5 + (g["cell_cen"] - 0.5) @ a  # in (0,1): every cell interfacial
    assert (F > 0).all() and (F < 1).all()
    st = om.taggrid(F)
    n = om.lsgir(st["F"], st["tag_c"], 1.5)
    assert np.allclose(n, a / np.linalg.norm(a), atol=1e-13)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_lsgir_axis_normal_for_an_axis_aligned_interface(orc, axis):
    """An interface plane x_axis = 0.43 on the uniform hex grid, with F the
    exact cell fractions: every interior interfacial cell's stencil is
    symmetric in the two other directions, where F is constant, so the LSGIR
    normal is the axis itself, pointing into the fluid (towards larger F, Sec.
    2.1.1), and the plane constant puts the plane at 0.43 exactly (Sec. 2.1).
    A transposed moment, a wrong sign of the normal or of the plane constant
    fails this."""
    n = 8
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    g = om.geometry()
    h = 1.0 / n
    x = g["cell_cen"][:, axis]
    F = np.clip((0.43 - (x - 0.5 * h)) / h, 0.0, 1.0)   # fluid where x_axis < 0.43
    st = om.reconstruct(F)
    inter = st["tag_c"] == 0
    lo = g["cell_cen"] - 0.5 * h
    interior = np.all((lo > 1e-12) & (lo + h < 1 - 1e-12), axis=1)
    sel = inter & interior
    assert sel.sum() == (n - 2) ** 2
    e = np.zeros(3)
    e[axis] = -1.0
    assert np.abs(st["nrm"][sel] - e).max() < 1e-14
    # plane n.(x - xc) + C = 0 at x_axis = 0.43: C = 0.43 - xc_axis
    assert np.abs(st["C"][sel] - (0.43 - x[sel])).max() < 1e-14


def test_lsgir_rotation_invariance(orc):
    m = I.kuhn_tet_mesh(3, seed=6)
    om = orc.Mesh(m)
    g = om.geometry()
    F = np.clip(0.5 + 3 * ((g["cell_cen"] - 0.45) ** 2).sum(1) - 0.2, 0.05, 0.95)
    st = om.taggrid(F)
    n = om.lsgir(st["F"], st["tag_c"], 1.5)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    m2 = dict(m)
    m2["X"] = m["X"] @ R.T
    om2 = orc.Mesh(m2)
    st2 = om2.taggrid(F)
    n2 = om2.lsgir(st2["F"], st2["tag_c"], 1.5)
    assert np.allclose(n2, n @ R.T, atol=1e-12)


# ---------------------------------------------------------------- NMFPA
def _nmfpa_faces(nI):
    """Faces of the non-matched polyhedron as Sec. 2.2.3 states them: the
    cell face, I side faces, the back-traced face (I+2 faces)."""
    faces = [list(range(nI))]
    faces += [[(i + 1) % nI, i, nI + i, nI + (i + 1) % nI] for i in range(nI)]
    faces.append([nI + i for i in range(nI - 1, -1, -1)])
    return faces


@pytest.mark.parametrize("gen", ["hex", "tet", "trihex"])
def test_nmfpa_is_the_prism_of_the_face_velocity(orc, gen):
    """Every vertex moves back by dt u(x_c, t^{n+1/2}) (the written-out
    rotation field at the face centre): the side faces are parallelograms,
    the back-traced face is the face's translate, and the volume of the
    I+2 faces equals V_d without any adjustment."""
    m = {"hex": lambda: I.hex_mesh(5), "tet": lambda: I.kuhn_tet_mesh(4, seed=5),
         "trihex": lambda: I.trihex_mesh(3, seed=2)}[gen]()
    om = orc.Mesh(m)
    g = om.geometry()
    omega, c = 2.0 * np.pi, (0.5, 0.5, 0.5)
    vel = I.rotation(omega, c)
    dt = 0.02
    for f in range(0, len(m["owner"]), 3):
        P, vd, fl = om.nmfpa(f, vel, 0.1, dt)
        X = _face_nodes(m, f)
        nI = len(X)
        assert P.shape[0] == 2 * nI and fl == 0
        uc = _rot_u(g["face_cen"][f][None, :], omega, c)[0]
        assert np.allclose(P[:nI], X, atol=1e-15)
        assert np.allclose(P[nI:], X - dt * uc, atol=1e-15)
        assert abs(vd - uc @ g["face_nrm"][f] * g["face_area"][f] * dt) < 1e-18
        vol = orc.poly_volume(P - X.mean(0), _nmfpa_faces(nI))
        A = g["face_area"][f]
        assert abs(vol - vd) <= 1e-14 * max(abs(vd), A ** 1.5), (f, vol, vd)


def test_nmfpa_and_fmfpa_agree_for_uniform_flow(orc):
    """A uniform field gives the same exact prism to every construction."""
    m = I.kuhn_tet_mesh(5, seed=8)
    om = orc.Mesh(m)
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.22), levels=3))
    vel = I.translation((0.4, -0.3, 0.2))
    dt = om.suggest_dt(vel, 0.0, 0.6, 10.0)
    Vd0, VF0, _ = om.faceflux(vel, 0.0, dt, st, orc.FMFPA)
    Vd2, VF2, s2 = om.faceflux(vel, 0.0, dt, st, orc.NMFPA)
    assert np.array_equal(Vd0, Vd2) and s2[1] == 0 and s2[2] == 0
    assert np.abs(VF2 - VF0).max() < 1e-15 * np.abs(Vd0).max() * 100


def test_nmfpa_cfl1_translation_shifts_exactly(orc):
    n = 6
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.45, 0.52, 0.48), 0.27), levels=3))
    new = om.step(I.translation((1.0, 0.0, 0.0)), 0.0, 1.0 / n, st, method=orc.NMFPA)
    F = st["F"].reshape(n, n, n)
    G = new["F_unclipped_cut"].reshape(n, n, n)
    assert np.abs(G[:, :, 1:] - F[:, :, :-1]).max() < 2e-15
    assert np.abs(G[:, :, 0]).max() == 0.0


def test_nmfpa_is_not_strictly_conservative(orc):
    """Sec. 4: NMFPA is not strictly conservative because the polyhedra of
    neighbouring faces overlap or leave gaps, so F leaves [0, 1] and the
    final clip removes volume; with the face-matched polyhedra the same
    rotation keeps the volume to rounding (the field is linear, so the
    discrete divergence vanishes and only the clip could change it)."""
    m = I.hex_mesh(16)
    om = orc.Mesh(m)
    V = om.geometry()["cell_vol"]
    F0 = I.init_fraction(m, I.sphere((0.5, 0.75, 0.5), 0.15), levels=3)
    vel = I.rotation(1.0, (0.5, 0.5, 0.5))
    loss = {}
    for meth in (orc.FMFPA, orc.NMFPA):
        st = om.reconstruct(F0)
        v0 = (V * st["F"]).sum()
        t, worst = 0.0, 0.0
        for _ in range(6):
            dt = om.suggest_dt(vel, t, 0.9, 100.0)
            vb = (V * st["F"]).sum()
            new = om.step(vel, t, dt, st, method=meth)
            worst = max(worst, abs((V * new["F_unclipped_cut"]).sum() - vb) / v0)
            st, t = new, t + dt
        loss[meth] = worst
    assert loss[orc.FMFPA] < 1e-13, loss
    assert loss[orc.NMFPA] > 1e-8, loss


def test_nmfpa_uses_the_midtime_face_velocity(orc):
    """Time-modulated deformation field (Sec. 4.2), written out: the shift
    of every vertex is dt u(x_c, t + dt/2)."""
    m = I.hex_mesh(4)
    om = orc.Mesh(m)
    T, t, dt = 3.0, 0.4, 0.05
    g = om.geometry()

    def u(x, tt):
        s_, s2 = np.sin(np.pi * x), np.sin(2 * np.pi * x)
        return np.cos(np.pi * tt / T) * np.array([2 * s_[0] ** 2 * s2[1] * s2[2],
                                                  -s2[0] * s_[1] ** 2 * s2[2],
                                                  -s2[0] * s2[1] * s_[2] ** 2])
    for f in range(0, len(m["owner"]), 5):
        P, _, _ = om.nmfpa(f, I.deformation(T), t + 0.5 * dt, dt)
        nI = P.shape[0] // 2
        assert np.allclose(P[nI:] - P[:nI], -dt * u(g["face_cen"][f], t + 0.5 * dt), atol=1e-16)


@pytest.mark.parametrize("method", ["FMFPA", "EMFPA", "NMFPA"])
def test_faceflux_monte_carlo(orc, method):
    """V_F of sample active faces (Sec. 2.2) against a Monte-Carlo integral of
    the fluid indicator (full cells 1, interfacial cells their PLIC half-
    space, empty cells 0; cells located on the uniform grid by index) times
    the winding number of the face's flux polyhedron (points and faces from
    the construction, written out here)."""
    n = 8
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.5, 0.55, 0.5), 0.27), levels=3))
    vel, t, dt = I.rotation(2 * np.pi), 0.0, 0.02
    meth = getattr(orc, method)
    Vd, VF, _ = om.faceflux(vel, t, dt, st, meth)
    g = om.geometry()
    build = {"FMFPA": (om.fmfpa, _fmfpa_faces), "EMFPA": (om.emfpa, _emfpa_faces),
             "NMFPA": (om.nmfpa, _nmfpa_faces)}[method]
    active = np.nonzero(st["tag_f"] == 0)[0]
    rng = np.random.default_rng(17)
    for f in rng.choice(active, 6, replace=False):
        P, vd, _ = build[0](int(f), vel, t + 0.5 * dt, dt)
        nI = {"FMFPA": (P.shape[0] - 1) // 2, "EMFPA": (P.shape[0] - 1) // 3,
              "NMFPA": P.shape[0] // 2}[method]
        tris = fan_tris(P, build[1](nI))
        lo, hi = P.min(0), P.max(0)
        N = 200000
        X = lo + (hi - lo) * rng.random((N, 3))
        w = winding_number(X, tris)
        ijk = np.clip(np.floor(X * n).astype(int), 0, n - 1)
        cell = ijk[:, 0] + n * (ijk[:, 1] + n * ijk[:, 2])
        tc = st["tag_c"][cell]
        side = np.einsum("ij,ij->i", st["nrm"][cell], X - g["cell_cen"][cell]) + st["C"][cell]
        fluid = (tc == 1) | ((tc == 0) & (side >= 0))
        box = np.prod(hi - lo)
        vals = w * fluid
        mc, sig = vals.mean() * box, vals.std() * box / np.sqrt(N)
        assert abs(VF[f] - mc) < 5 * sig + 1e-12, (method, f, VF[f], mc, sig)


# ---------------------------------------------------------------- LSFIR
def _ang(a, b):
    """angle between unit vectors, accurate near 0"""
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def test_plic_centre_closed_forms(orc):
    """Vertex average of the PLIC polygon of the unit cube (Sec. 2.1.2): a
    plane x = 0.3 gives a square centred at (0.3, 1/2, 1/2); x + y + z = s < 1
    cuts a corner triangle centred at (s/3, s/3, s/3); x = 1 contains a face,
    whose four vertices are the polygon's."""
    om = orc.Mesh(I.hex_mesh(1))
    # plane n.(x - xc) + C = 0 with xc = (1/2, 1/2, 1/2)
    out, k = om.plic_centre(0, [1.0, 0.0, 0.0], 0.5 - 0.3)
    assert k == 4 and np.allclose(out, [0.3, 0.5, 0.5], atol=1e-15)
    n = np.ones(3) / np.sqrt(3.0)
    for s_ in (0.2, 0.7):  # x + y + z = s  <=>  C = (1.5 - s) / sqrt(3)
        for sign in (1.0, -1.0):  # either side may be the fluid
            out, k = om.plic_centre(0, sign * n, sign * (1.5 - s_) / np.sqrt(3.0))
            assert k == 3 and np.allclose(out, [s_ / 3] * 3, atol=1e-15), (s_, k, out)
    # the plane x = 1 through a whole face: phi is exactly 0 at its four
    # vertices (C formed from the centroid as the oracle forms phi), which
    # are the polygon's vertices, each once
    xc = om.geometry()["cell_cen"][0]
    out, k = om.plic_centre(0, [1.0, 0.0, 0.0], -(1.0 - xc[0]))
    assert k == 4 and np.array_equal(out, [1.0, 0.5, 0.5]), (k, out)


def _exact_plane_F(om, nrm, p0):
    g = om.geometry()
    return np.array([om.cell_cut_volume(c, nrm, nrm @ (g["cell_cen"][c] - p0))
                     for c in range(om.n_cell)]) / g["cell_vol"]


@pytest.mark.parametrize("gen", ["hex", "tet", "trihex"])
def test_lsfir_reproduces_a_plane(orc, gen):
    """A planar interface: if every interfacial cell carries the exact plane,
    the PLIC centres lie on it and one least-squares update returns the
    plane's normal (the fixed point of Sec. 2.1.2)."""
    m = {"hex": lambda: I.hex_mesh(6), "tet": lambda: I.kuhn_tet_mesh(5, seed=3),
         "trihex": lambda: I.trihex_mesh(4, seed=2)}[gen]()
    om = orc.Mesh(m)
    nt = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    p0 = np.array([0.5, 0.48, 0.52])
    st = om.taggrid(_exact_plane_F(om, nt, p0))
    band = st["tag_c"] == 0
    N = np.tile(nt, (om.n_cell, 1))
    Ce = om.plane_constant(st["F"], st["tag_c"], N)
    xp = om.geometry()["cell_cen"].copy()
    for c in np.nonzero(band)[0]:
        xp[c] = om.plic_centre(c, nt, Ce[c])[0]
    assert np.abs((xp[band] - p0) @ nt).max() < 1e-11
    cand, kept = om.lsfir_normals(st["tag_c"], N, xp)
    assert kept == 0
    assert _ang(cand[band], nt).max() < 1e-9


def test_lsfir_normal_minimises_H_bruteforce(orc):
    """For sample cells the update equals a direct minimisation of
    H = sum w_k (n.(x_k - x))^2, w_k = |x_k - x|^-2.5, over unit vectors, with
    the valid neighbours (interfacial, previous normals within 45 degrees)
    chosen here from the neighbour lists."""
    m = I.kuhn_tet_mesh(5, seed=12)
    om = orc.Mesh(m)
    st = om.taggrid(I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.3), levels=3))
    tc = st["tag_c"]
    ng = om.lsgir(st["F"], tc)
    Cg = om.plane_constant(st["F"], tc, ng)
    xp = om.geometry()["cell_cen"].copy()
    band = np.nonzero(tc == 0)[0]
    for c in band:
        xp[c] = om.plic_centre(c, ng[c], Cg[c])[0]
    cand, _ = om.lsfir_normals(tc, ng, xp)
    ptr, idx = om.neighbors()
    # unit vectors: a Fibonacci sphere, then local refinement
    k = np.arange(20000) + 0.5
    th, ph = np.arccos(1 - 2 * k / k.size), np.pi * (1 + 5 ** 0.5) * k
    U = np.stack([np.cos(ph) * np.sin(th), np.sin(ph) * np.sin(th), np.cos(th)], 1)
    checked = 0
    for c in band[::7]:
        nb = [q for q in idx[ptr[c]:ptr[c + 1]] if tc[q] == 0 and ng[c] @ ng[q] > np.sqrt(0.5)]
        if len(nb) < 3:
            continue
        D = xp[nb] - xp[c]
        w = np.linalg.norm(D, axis=1) ** -2.5
        H = lambda V: ((V @ D.T) ** 2 * w).sum(-1)
        best = U[np.argmin(H(U))]
        for step in (2e-2, 5e-3, 1e-3, 2e-4, 5e-5, 1e-5):
            for _ in range(60):
                trial = best + step * np.random.default_rng(int(c)).normal(size=(64, 3))
                trial /= np.linalg.norm(trial, axis=1, keepdims=True)
                j = np.argmin(H(trial))
                if H(trial[j]) < H(best):
                    best = trial[j]
        if best @ ng[c] < 0:
            best = -best
        assert _ang(cand[c], best) < 1e-4, (c, cand[c], best)
        checked += 1
    assert checked >= 10


def test_lsfir_acceptance_limit(orc):
    """Outer iteration (Sec. 2.1.2): a change is accepted only below
    30 degrees / I_out. On a planar interface, one cell's normal turned by 20
    degrees is corrected in the first iteration; turned by 40 degrees (still a
    valid neighbour, < 45) its candidate is refused in every iteration."""
    m = I.trihex_mesh(4, seed=2)
    om = orc.Mesh(m)
    nt = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    st = om.taggrid(_exact_plane_F(om, nt, np.array([0.5, 0.48, 0.52])))
    band = np.nonzero(st["tag_c"] == 0)[0]
    F = st["F"]
    c0 = band[np.argmin(np.abs(F[band] - 0.5))]  # a well-filled cell
    axis = np.cross(nt, [1.0, 0.0, 0.0])
    axis /= np.linalg.norm(axis)
    for deg, fixed in ((20.0, True), (40.0, False)):
        a = np.radians(deg)
        turned = nt * np.cos(a) + np.cross(axis, nt) * np.sin(a)
        N0 = np.tile(nt, (om.n_cell, 1))
        N0[c0] = turned
        nf, Cf, it = om.lsfir(F, st["tag_c"], N0, n_out=4, tol=1e-3)
        if fixed:
            assert _ang(nf[c0], nt) < 1e-3, deg
        else:
            assert _ang(nf[c0], turned) == 0.0, deg
        others = np.setdiff1d(band, [c0])
        assert _ang(nf[others], nt).max() < 0.05


def test_lsfir_acceptance_limit_shrinks_with_the_iteration(orc):
    """A candidate turning a normal by 20 degrees is taken in outer
    iteration 1 (limit 30) and refused in iteration 2 (limit 15); 10 degrees
    is taken in 1, 2 and 3 (limit 10 is strict) is refused; non-interfacial
    cells never change (Sec. 2.1.2)."""
    om = orc.Mesh(I.hex_mesh(2))
    tags = np.array([0, 0, 0, 0, 0, 0, 1, -1], np.int8)
    prev = np.tile([0.0, 0.0, 1.0], (8, 1))

    def turned_by(deg):
        a = np.radians(deg)
        return np.array([np.sin(a), 0.0, np.cos(a)])
    degs = [20.0, 10.0, 10.0, 9.9, 29.9, 30.1, 5.0, 5.0]
    cand = np.array([turned_by(d) for d in degs])
    took = {}
    for io in (1, 2, 3):
        new, t = om.lsfir_accept(tags, io, cand, prev)
        took[io] = [bool(np.array_equal(new[c], cand[c])) for c in range(8)]
        assert all(np.array_equal(new[c], prev[c]) for c in range(8) if not took[io][c])
        acc = [degs[c] for c in range(8) if took[io][c]]
        assert abs(t - np.radians(max(acc))) < 1e-12
    assert took[1] == [True, True, True, True, True, False, False, False]
    assert took[2] == [False, True, True, True, False, False, False, False]
    assert took[3] == [False, False, False, True, False, False, False, False]


def _renumber_cells(m, perm):
    """the same mesh with cell c renamed perm[c]; a face whose owner would
    get the larger index is flipped so that it still leaves its owner"""
    own, nbr = perm[m["owner"]], np.where(m["neighbour"] >= 0, perm[np.maximum(m["neighbour"], 0)], -1)
    fp, fv = m["face_ptr"], m["face_vert"].copy()
    flip = (nbr >= 0) & (nbr < own)
    for f in np.nonzero(flip)[0]:
        fv[fp[f]:fp[f + 1]] = fv[fp[f]:fp[f + 1]][::-1]
    o2 = np.where(flip, nbr, own).astype(np.int32)
    n2 = np.where(flip, own, nbr).astype(np.int32)
    return {"X": m["X"], "face_ptr": fp, "face_vert": fv, "owner": o2, "neighbour": n2,
            "n_cell": m["n_cell"]}


def test_lsfir_is_independent_of_cell_order(orc):
    """Every cell's new orientation is computed from the previous iteration's
    planes before any is updated (Sec. 2.1.2), so renumbering the cells
    renumbers the result and changes nothing else."""
    m = I.kuhn_tet_mesh(4, seed=21)
    om = orc.Mesh(m)
    F = I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.3), levels=3)
    st = om.reconstruct(F, recon=orc.LSFIR)
    perm = np.random.default_rng(5).permutation(m["n_cell"])
    m2 = _renumber_cells(m, perm)
    F2 = np.empty_like(F)
    F2[perm] = F
    st2 = orc.Mesh(m2).reconstruct(F2, recon=orc.LSFIR)
    band = np.nonzero(st["tag_c"] == 0)[0]
    assert np.array_equal(st2["tag_c"][perm], st["tag_c"])
    assert np.abs(st2["nrm"][perm[band]] - st["nrm"][band]).max() < 1e-10
    assert np.abs(st2["C"][perm[band]] - st["C"][band]).max() < 1e-10
    assert st2["lsfir_iters"] == st["lsfir_iters"]


def test_lsfir_more_accurate_than_lsgir_and_converges(orc):
    """Sphere on jittered tets: the LSFIR normals (Sec. 2.1.2) are closer to
    the exact normal at the PLIC centre than the LSGIR ones, and the mean
    error falls by more than 1.6 when h halves."""
    ctr, R = np.array((0.5, 0.52, 0.48)), 0.3
    errs = []
    for n in (12, 24):
        m = I.kuhn_tet_mesh(n, seed=3)
        om = orc.Mesh(m)
        st = om.taggrid(I.init_fraction(m, I.sphere(ctr, R), levels=5))
        ng = om.lsgir(st["F"], st["tag_c"])
        Cg = om.plane_constant(st["F"], st["tag_c"], ng)
        nf, Cf, it = om.lsfir(st["F"], st["tag_c"], ng)
        band = np.nonzero(st["tag_c"] == 0)[0]

        def mean_err(N, Cc):
            e = []
            for c in band:
                xp = om.plic_centre(c, N[c], Cc[c])[0]
                e.append(_ang(N[c], -(xp - ctr) / np.linalg.norm(xp - ctr)))
            return float(np.mean(e))
        eg, ef = mean_err(ng, Cg), mean_err(nf, Cf)
        assert ef < 0.6 * eg, (n, ef, eg)
        errs.append(ef)
    assert errs[0] / errs[1] > 1.6, errs


def test_lsfir_rotation_invariance(orc):
    m = I.kuhn_tet_mesh(4, seed=6)
    om = orc.Mesh(m)
    x = om.geometry()["cell_cen"]
    # smooth and nowhere flat (no zero gradient, every cell interfacial)
    F = 0.5 + 0.25 * np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]) + 0.1 * x[:, 2]
    st = om.reconstruct(F, recon=orc.LSFIR)
    R = np.array([[math.cos(0.7), -math.sin(0.7), 0], [math.sin(0.7), math.cos(0.7), 0], [0, 0, 1]])
    m2 = dict(m)
    m2["X"] = m["X"] @ R.T
    st2 = orc.Mesh(m2).reconstruct(F, recon=orc.LSFIR)
    band = st["tag_c"] == 0
    assert np.allclose(st2["nrm"][band], st["nrm"][band] @ R.T, atol=1e-9)
    assert np.allclose(st2["C"][band], st["C"][band], atol=1e-9)


# ---------------------------------------------------------------- initfgrid
@pytest.mark.parametrize("gen", ["hex", "tet", "trihex"])
def test_initfgrid_halfspace_is_exact(orc, gen):
    """A planar surface is its own linear interpolant: the refinement gives
    every cell's exact cut volume (Sec. 2.1 closed forms pin the cut
    volume), for convex and non-convex cells alike."""
    m = {"hex": lambda: I.hex_mesh(5), "tet": lambda: I.kuhn_tet_mesh(4, seed=2),
         "trihex": lambda: I.trihex_mesh(3, seed=4)}[gen]()
    om = orc.Mesh(m)
    g = om.geometry()
    nt = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    p0 = np.array([0.5, 0.48, 0.52])
    F = om.initfgrid(I.shape_halfspace(p0, nt), 3)
    # fluid a.(x - p0) < 0: the cut volume of the plane with normal -a
    ex = np.array([om.cell_cut_volume(c, -nt, -nt @ (g["cell_cen"][c] - p0))
                   for c in range(om.n_cell)]) / g["cell_vol"]
    assert np.abs(F - ex).max() < 1e-13
    assert ((F > 0) & (F < 1)).sum() > 10


@pytest.mark.parametrize("shape", ["sphere", "cylinder"])
def test_initfgrid_converges_at_second_order(orc, shape):
    """Total fluid volume against the body's closed-form volume: the piecewise
    linear interpolant errs by O((h/ndiv)^2), so doubling ndiv divides the
    error by about four; cells away from the surface are exactly 0 or 1."""
    m = I.hex_mesh(12)
    om = orc.Mesh(m)
    V = om.geometry()["cell_vol"]
    if shape == "sphere":
        sh, exact = I.shape_sphere((0.5, 0.52, 0.48), 0.3), 4.0 / 3.0 * np.pi * 0.3 ** 3
    else:  # axis along y through the whole domain (the 2D test's cylinder, Sec. 4)
        sh, exact = I.shape_cylinder((0.5, 0.0, 0.55), (0.0, 1.0, 0.0), 0.25), np.pi * 0.25 ** 2
    err = []
    for n in (4, 8, 16):
        F = om.initfgrid(sh, n)
        assert F.min() >= 0 and F.max() <= 1
        err.append((V * F).sum() - exact)
    assert 3.3 < err[0] / err[1] < 4.7 and 3.3 < err[1] / err[2] < 4.7, err
    assert abs(err[2]) < 1e-4 * exact
    x = om.geometry()["cell_cen"]
    far = np.abs(np.linalg.norm((x - sh.c) * ([1, 0, 1] if shape == "cylinder" else 1), axis=1)
                 - sh.r) > 0.1
    F = om.initfgrid(sh, 4)
    assert set(np.unique(F[far])) <= {0.0, 1.0}


# ---------------------------------------------------------------- quasi-2D
def test_slab_geometry_closed_form(orc):
    """n x 1 x n cells on the unit cube (the 2D tests' grids, Sec. 4.3)."""
    n = 6
    m = I.slab_mesh(n)
    om = orc.Mesh(m)
    g = om.geometry()
    assert om.n_cell == n * n
    assert np.allclose(g["cell_vol"], 1.0 / n ** 2, rtol=1e-14)
    i, k = np.arange(n * n) % n, np.arange(n * n) // n
    assert np.allclose(g["cell_cen"], np.stack([(i + 0.5) / n, 0.5 + 0 * i, (k + 0.5) / n], 1),
                       atol=1e-15)
    # every cell is closed: the outward face vectors sum to zero
    A = g["face_nrm"] * g["face_area"][:, None]
    S = np.zeros((om.n_cell, 3))
    np.add.at(S, m["owner"], A)
    inner = m["neighbour"] >= 0
    np.add.at(S, m["neighbour"][inner], -A[inner])
    assert np.abs(S).max() < 1e-15
    # node neighbours: 8 inside, 3 at a corner
    ptr, idx = om.neighbors()
    cnt = np.diff(ptr)
    assert cnt.max() == 8 and cnt.min() == 3


def test_lsgir_quasi2d_pseudo_inverse(orc):
    """On a slab every neighbour offset has dy = 0, so the LSGIR system of
    Sec. 2.1.1 is singular; the minimum-norm least-squares solution recovers
    a linear field's in-plane gradient exactly, and drops a y-gradient the
    stencil cannot see."""
    m = I.slab_mesh(8)
    om = orc.Mesh(m)
    x = om.geometry()["cell_cen"]
    for a in ([0.3, 0.0, -0.4], [0.3, 0.25, -0.4], [-0.05, 0.0, 0.6]):
        a = np.array(a)
        st = om.taggrid(0.5 + (x - 0.5) @ a)
        n = om.lsgir(st["F"], st["tag_c"])
        band = st["tag_c"] == 0
        e = a * [1, 0, 1]
        assert band.sum() > 10
        assert np.abs(n[band] - e / np.linalg.norm(e)).max() < 1e-13, a


def test_deformation2d_field(orc):
    """The 2D deformation field of Sec. 4.3 at hand-evaluated points, its zero
    divergence and its zero y-component."""
    om = orc.Mesh(I.slab_mesh(2))
    vel = I.deformation2d(8.0)
    # x = z = 1/4: sin^2 = 1/2, sin cos = 1/2 -> u = -1/2, w = 1/2 (times cos(pi t/8))
    assert np.allclose(om.velocity(vel, [0.25, 0.3, 0.25], 0.0), [-0.5, 0.0, 0.5], atol=1e-15)
    assert np.allclose(om.velocity(vel, [0.25, 0.7, 0.25], 8.0 / 3.0), [-0.25, 0.0, 0.25], atol=1e-15)
    # x = 1/2, z = 1/4: u = -2 * 1 * 1/2 = -1, w = 2 * 1/2 * 0 = 0
    assert np.allclose(om.velocity(vel, [0.5, 0.1, 0.25], 0.0), [-1.0, 0.0, 0.0], atol=1e-15)
    rng = np.random.default_rng(4)
    h = 1e-5
    for X in rng.random((20, 3)):
        div = 0.0
        for d in range(3):
            e = np.zeros(3); e[d] = h
            div += (om.velocity(vel, X + e, 1.0)[d] - om.velocity(vel, X - e, 1.0)[d]) / (2 * h)
        assert abs(div) < 1e-8
        assert om.velocity(vel, X, 1.0)[1] == 0.0


def test_deformation2d_on_slab_conserves_and_stays_2d(orc):
    """A few steps of the 2D deformation test on a slab: the y-faces carry
    nothing, the volume is conserved (zero divergence, the body away from the
    walls), and F stays between 0 and 1."""
    m = I.slab_mesh(24)
    om = orc.Mesh(m)
    V = om.geometry()["cell_vol"]
    st = om.reconstruct(om.initfgrid(I.shape_cylinder((0.5, 0.0, 0.75), (0, 1, 0), 0.15), 10))
    vel = I.deformation2d(8.0)
    ny = np.abs(om.geometry()["face_nrm"][:, 1]) > 0.5
    t = 0.0
    for _ in range(4):
        dt = om.suggest_dt(vel, t, 0.5, 8.0)
        v0 = (V * st["F"]).sum()
        new = om.step(vel, t, dt, st)
        assert np.all(new["Vd"][ny] == 0.0) and np.all(new["VF"][ny] == 0.0)
        assert abs((V * new["F_unclipped_cut"]).sum() - v0) < 1e-13 * v0
        st, t = new, t + dt


# ---------------------------------------------------------------- whole step
def test_cfl1_translation_shifts_exactly(orc):
    """u = (1,0,0), dt = h on a uniform grid: every x-face flux polyhedron is
    exactly the upstream cell, so F moves one cell per step for ANY F."""
    n = 6
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    g = om.geometry()
    F0 = I.init_fraction(m, I.sphere((0.45, 0.52, 0.48), 0.27), levels=3)
    st = om.reconstruct(F0)
    vel = I.translation((1.0, 0.0, 0.0))
    new = om.step(vel, 0.0, 1.0 / n, st)
    F = st["F"].reshape(n, n, n)      # [k, j, i]
    G = new["F_unclipped_cut"].reshape(n, n, n)
    assert np.abs(G[:, :, 1:] - F[:, :, :-1]).max() < 2e-15
    assert np.abs(G[:, :, 0]).max() == 0.0


@pytest.mark.parametrize("method", ["FMFPA", "EMFPA", "NMFPA"])
@pytest.mark.parametrize("frac", [0.5, 0.3])
def test_planar_interface_translates_exactly(orc, method, frac):
    """A planar interface x = 0.43 (fluid behind it, exact cell fractions) in
    the uniform flow u = (1, 0, 0) at a CFL below 1: PLIC represents the plane
    exactly (Sec. 2.1) and every construction gives the exact prism of the
    face in uniform flow (Sec. 2.2), so after one step F holds the exact
    fractions of the plane at x = 0.43 + dt, up to rounding. Cells next to the
    inflow wall x = 0 are left out: no fluid enters from outside the domain."""
    n = 8
    h = 1.0 / n
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    x = om.geometry()["cell_cen"][:, 0]
    F0 = np.clip((0.43 - (x - 0.5 * h)) / h, 0.0, 1.0)
    st = om.reconstruct(F0)
    dt = frac * h
    new = om.step(I.translation((1.0, 0.0, 0.0)), 0.0, dt, st, method=getattr(orc, method))
    exact = np.clip((0.43 + dt - (x - 0.5 * h)) / h, 0.0, 1.0)
    keep = x > 1.5 * h
    assert np.abs(new["F"][keep] - exact[keep]).max() < 1e-14


def test_translation_vdt_zero_and_conservation(orc):
    m = I.kuhn_tet_mesh(5, seed=8)
    om = orc.Mesh(m)
    g = om.geometry()
    F0 = I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.22), levels=3)
    st = om.reconstruct(F0)
    vel = I.translation((0.4, -0.3, 0.2))
    dt = om.suggest_dt(vel, 0.0, 0.4, 10.0)
    Vd, VF, stats = om.faceflux(vel, 0.0, dt, st)
    # uniform field: sum of sigma V_d over each closed cell vanishes
    vdt = np.zeros(om.n_cell)
    np.add.at(vdt, m["owner"], Vd)
    inner = m["neighbour"] >= 0
    np.add.at(vdt, m["neighbour"][inner], -Vd[inner])
    assert np.abs(vdt).max() < 1e-17
    # the body stays away from the boundary: total volume conserved
    F1 = om.vofadv(st["F"], Vd, VF)
    V = g["cell_vol"]
    assert abs((V * F1).sum() - (V * st["F"]).sum()) < 1e-15 * (V * st["F"]).sum()
    assert F1.min() >= 0 and F1.max() <= 1


def test_deformation_conserves_volume(orc):
    m = I.hex_mesh(16)
    om = orc.Mesh(m)
    V = om.geometry()["cell_vol"]
    st = om.reconstruct(I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15)))
    vel = I.deformation(3.0)
    t = 0.0
    for _ in range(5):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        v0 = (V * st["F"]).sum()
        new = om.step(vel, t, dt, st)
        G = new["F_unclipped_cut"]
        # E_bound of this step is tiny and the body never touches the wall
        assert abs((V * G).sum() - v0) < 1e-13 * v0
        st, t = new, t + dt


def test_step_count_matches_paper(orc):
    """Eq. eq:cfl with the time-modulated field gives about 24/(pi h) steps
    to t = 3 at CFL 0.5; the paper's tables imply the same count."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "step_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for grid, _, _, steps in rows:
        pred = 24.0 / (math.pi / int(grid))
        assert abs(pred - int(steps)) / int(steps) < 0.05
    n = 16
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    vel = I.deformation(3.0)
    t, k = 0.0, 0
    while t < 3.0 - 1e-12:
        t += om.suggest_dt(vel, t, 0.5, 3.0)
        k += 1
    assert abs(k - 24.0 * n / math.pi) / (24.0 * n / math.pi) < 0.03


@pytest.mark.parametrize("grid", ["hex", "tets", "trihex"])
@pytest.mark.parametrize("method", ["FMFPA", "EMFPA", "NMFPA"])
@pytest.mark.parametrize("cfl", [0.5, 0.8, 1.0])
def test_candidate_cells_cover_the_flux_polyhedron(orc, grid, method, cfl):
    """The candidate cells of a face (the node neighbours of its owner and of
    its neighbour, with the two cells themselves) cover its flux polyhedron
    (Sec. 2.2: the donating region may span several cells). With every cell
    full and every face evaluated geometrically, the truncation sums
    vol(polyhedron ∩ cell) over the candidates, which must then equal the
    polyhedron's own signed volume V_d. Faces with a node on the domain
    boundary are left out: their polyhedra may reach outside the domain,
    where there is no fluid (NMFPA's translated prism does so even where the
    wall-normal velocity vanishes). Interior faces are covered at CFL 0.5 on
    every grid (the jittered workloads run at 0.4 and 0.5) and up to CFL 1 on
    the uniform hex grid; on the jittered grids at CFL 0.8 a few polyhedra
    already reach past the ring (the CFL bound uses cell bounding boxes,
    which overstate the size of a jittered cell in the direction of flow), so
    those cases are not pins. A candidate set missing a ring, or a
    truncation that drops or doubles a piece, fails this."""
    if cfl > 0.5 and grid != "hex":
        pytest.skip("above CFL 0.5 the ring covers the polyhedra only on the uniform grid")
    if grid == "hex":
        m = I.hex_mesh(6)
    elif grid == "tets":
        m = I.kuhn_tet_mesh(4, seed=4)
    else:
        m = I.trihex_mesh(4, seed=2)
    if method == "EMFPA" and np.diff(m["face_ptr"]).max() > 6:
        pytest.skip("EMFPA takes faces of up to 6 nodes")
    om = orc.Mesh(m)
    nc, nf = om.n_cell, om.n_face
    st = {"F": np.ones(nc), "tag_f": np.zeros(nf, np.int8), "tag_c": np.ones(nc, np.int8),
          "nrm": np.zeros((nc, 3)), "C": np.zeros(nc)}
    vel, t = I.deformation(3.0), 0.3
    dt = om.suggest_dt(vel, t, cfl, 1e9)
    Vd, VF, _ = om.faceflux(vel, t, dt, st, method=getattr(orc, method))
    V = om.geometry()["cell_vol"]
    X, fv, fp = m["X"], m["face_vert"], m["face_ptr"]
    inner = np.array([not np.any((X[fv[fp[f]:fp[f + 1]]] < 1e-12) |
                                 (X[fv[fp[f]:fp[f + 1]]] > 1 - 1e-12)) for f in range(nf)])
    scale = V[m["owner"]][inner]
    assert inner.sum() >= 100
    assert np.abs(Vd[inner]).max() > 0.05 * scale.max()  # the polyhedra are not trivial
    assert (np.abs(VF - Vd)[inner] / scale).max() < 1e-13

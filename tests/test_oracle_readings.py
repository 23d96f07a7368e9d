"""Pins of three readings of the paper that fix numbers the other pins leave
free, each with planted mistakes that must fail it.

- LSGIR weights (Sec. 2.1.1, Eqs. eq:lsgir1, eq:lsgir2, lsgir-beta): the
  normal of a cell whose 26-cell stencil sees a field with a cubic cross term
  has a direction that depends on the exponent beta, on the squaring of the
  weights in the normal equations and on the stencil's edge and corner
  neighbours; on the uniform hex grid it is a closed form in h, sqrt(2) h and
  sqrt(3) h.
- FMFPA back-trace (Sec. 2.2.2): each back-traced vertex lies on
  the two side planes that meet at its face node (each side plane contains
  its edge and is parallel to the velocity at the edge centre), and it is the
  orthogonal projection of the streak-line point x_i - dt u(x_i) (Eq.
  streak-line2) on their line of intersection: the residual from that point
  is perpendicular to the line. Checked in rigid rotation and in the
  time-modulated Enright field, written out here, at t + dt/2.
- IDW node values (Sec. 3.3): a hand-computed F* at the centre
  node of a 2 x 2 x 2 grid whose cells have different widths.

A planted mistake is a one-line change of oracle.c compiled into a separate
library (the product is never involved); the pin must fail with it.
"""
import importlib.util
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")


def mutant(tmp_path, old, new, tag):
    """The oracle package with `old` replaced by `new` in oracle.c (exactly
    one occurrence), compiled with the oracle's own flags into tmp_path."""
    src = open(os.path.join(ORACLE_DIR, "oracle.c")).read()
    assert src.count(old) == 1, old
    d = tmp_path / tag
    d.mkdir()
    (d / "oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE_DIR, "oracle.h"), d / "oracle.h")
    so = str(d / "liboracle_mut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", "-o", so, str(d / "oracle.c"), "-lm"], check=True)
    spec = importlib.util.spec_from_file_location(f"oracle_mut_{tag}",
                                                  os.path.join(ORACLE_DIR, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._LIB = so
    mod._lib = None
    mod.build = lambda force=False: so
    return mod


# ------------------------------------------------------------- LSGIR weights
def lsgir_direction(beta):
    """Direction of the LSGIR gradient at an interior cell of a uniform hex
    grid for Delta F = s (X + Y (X^2 + Z^2)), X, Y, Z the offsets of the
    neighbour in units of h. The 26-cell stencil is symmetric under each
    axis reflection, so A^T A is diagonal with equal entries
    D = sum w^2 d_x^2, and A^T b = s (D, N, 0) with
    N = sum w^2 d_y^2 (d_x^2 + d_z^2) / h^2, w^2 = |d|^(-2 beta):
    the 2 face neighbours along y contribute 0 to N, the 8 edge neighbours
    with d_y != 0 ... counted by distance class (h, sqrt2 h, sqrt3 h):
      D / h^(2-2b) = 2 * 1 + 8 * 2^-b + 8 * 3^-b
      N / h^(2-2b) = 8 * 2^-b * 1 + 8 * 3^-b * 2   (edge: one of d_x, d_z
      nonzero; corner: both)."""
    D = 2.0 + 8.0 * 2.0 ** -beta + 8.0 * 3.0 ** -beta
    N = 8.0 * 2.0 ** -beta + 16.0 * 3.0 ** -beta
    v = np.array([D, N, 0.0])
    return v / np.linalg.norm(v)


def _lsgir_case(orc, beta):
    n = 8
    m = I.hex_mesh(n)
    om = orc.Mesh(m)
    g = om.geometry()
    h = 1.0 / n
    x0 = np.array([3.5, 3.5, 3.5]) * h
    c = int(np.argmin(np.abs(g["cell_cen"] - x0).sum(1)))
    X, Y, Z = ((g["cell_cen"] - x0) / h).T
    F = 0.5 + 0.02 * (X + Y * (X ** 2 + Z ** 2))
    nrm = om.lsgir(F, np.zeros(m["n_cell"], np.int8), beta)
    return nrm[c]


@pytest.mark.parametrize("beta", [1.5, 2.0])
def test_lsgir_weights_closed_form(orc, beta):
    got = _lsgir_case(orc, beta)
    assert np.abs(got - lsgir_direction(beta)).max() < 1e-13, (got, lsgir_direction(beta))


def test_lsgir_closed_form_separates_the_readings():
    """The closed form distinguishes the readings a mistake would produce:
    beta 2 instead of 1.5, weights not squared (beta / 2), face neighbours
    only (N = 0), no corner neighbours."""
    ref = lsgir_direction(1.5)
    face_only = np.array([1.0, 0.0, 0.0])
    b = 1.5
    no_corner = np.array([2.0 + 8.0 * 2.0 ** -b, 8.0 * 2.0 ** -b, 0.0])
    no_corner /= np.linalg.norm(no_corner)
    for other in (lsgir_direction(2.0), lsgir_direction(0.75), face_only, no_corner):
        assert np.abs(other - ref).max() > 1e-2


LSGIR_MISTAKES = {
    "beta_fixed_2": ("double w = pow(norm3(d), -beta); /* Eq. lsgir-beta */",
                     "double w = pow(norm3(d), -2.0);"),
    "weights_not_squared": ("double w2 = w * w;", "double w2 = w;"),
    "face_neighbours_only": ("      double w = pow(norm3(d), -beta); /* Eq. lsgir-beta */",
                             "      if ((d[0] != 0) + (d[1] != 0) + (d[2] != 0) > 1) continue;\n"
                             "      double w = pow(norm3(d), -beta);"),
    "no_corner_neighbours": ("      double w = pow(norm3(d), -beta); /* Eq. lsgir-beta */",
                             "      if (d[0] != 0 && d[1] != 0 && d[2] != 0) continue;\n"
                             "      double w = pow(norm3(d), -beta);"),
}


@pytest.mark.parametrize("name", sorted(LSGIR_MISTAKES))
def test_lsgir_pin_catches_planted_mistake(tmp_path, name):
    old, new = LSGIR_MISTAKES[name]
    mut = mutant(tmp_path, old, new, name)
    got = _lsgir_case(mut, 1.5)
    assert np.abs(got - lsgir_direction(1.5)).max() > 1e-6, name


# ------------------------------------------------------------- FMFPA back-trace
def _deform_u(x, tt, T=3.0):
    """Enright deformation field of Sec. 4.2 with period T, written out"""
    s, s2 = np.sin(np.pi * x), np.sin(2 * np.pi * x)
    gt = np.cos(np.pi * tt / T)
    return gt * np.stack([2 * s[:, 0] ** 2 * s2[:, 1] * s2[:, 2],
                          -s2[:, 0] * s[:, 1] ** 2 * s2[:, 2],
                          -s2[:, 0] * s2[:, 1] * s[:, 2] ** 2], 1)


def _rot_u(x, tt, omega=2 * np.pi, c=(0.5, 0.5, 0.5)):
    return np.stack([-omega * (x[:, 1] - c[1]), omega * (x[:, 0] - c[0]), 0.0 * x[:, 2]], 1)


def _backtrace_residuals(om, m, vel, ufun, t, dt):
    """Largest violations, over the faces, of: back-traced vertex on side
    plane i-1 and on side plane i; residual from the streak-line point
    perpendicular to their line. Relative to |dt u| (the displacement)."""
    th = t + 0.5 * dt
    worst, checked = 0.0, 0
    fp, fv = m["face_ptr"], m["face_vert"]
    for f in range(0, len(m["owner"]), 2):
        P, vd, fl = om.fmfpa(f, vel, th, dt)
        if fl & 1:
            continue  # ill-conditioned side planes: the streak-line point itself is used
        X = m["X"][fv[fp[f]:fp[f + 1]]]
        nI = len(X)
        uv = ufun(X, th)
        ue = ufun(0.5 * (X + np.roll(X, -1, 0)), th)
        s = np.cross(np.roll(X, -1, 0) - X, ue)        # side plane normals
        xb = P[nI:2 * nI]
        scale = dt * np.linalg.norm(uv, axis=1).max() + 1e-300
        for i in range(nI):
            im = (i - 1) % nI
            if np.linalg.norm(s[i]) == 0.0 or np.linalg.norm(s[im]) == 0.0:
                continue  # no side plane (edge velocity zero)
            dx = xb[i] - X[i]
            dirn = np.cross(s[im], s[i])
            dirn /= np.linalg.norm(dirn)
            on_i = abs(np.dot(s[i], dx)) / np.linalg.norm(s[i])
            on_im = abs(np.dot(s[im], dx)) / np.linalg.norm(s[im])
            perp = abs(np.dot(X[i] - dt * uv[i] - xb[i], dirn))
            worst = max(worst, on_i / scale, on_im / scale, perp / scale)
        checked += 1
    assert checked > 20
    return worst


@pytest.mark.parametrize("field", ["rotation", "deformation"])
@pytest.mark.parametrize("gen", ["hex", "tet"])
def test_fmfpa_backtrace_reading(orc, field, gen):
    m = I.hex_mesh(5) if gen == "hex" else I.kuhn_tet_mesh(3, seed=5)
    om = orc.Mesh(m)
    if field == "rotation":
        vel, ufun, t = I.rotation(2 * np.pi), _rot_u, 0.1
    else:
        vel, ufun, t = I.deformation(3.0), _deform_u, 0.4
    assert _backtrace_residuals(om, m, vel, ufun, t, 0.04) < 1e-11


FMFPA_MISTAKES = {
    "edge_velocity_in_projection": ("double k = dt * dot3(uv[i], d) / dd;",
                                    "double k = dt * dot3(ue[i], d) / dd;"),
    "streak_point_no_projection": ("for (int q = 0; q < 3; ++q) xb[i][q] = x[i][q] - k * d[q];",
                                   "for (int q = 0; q < 3; ++q) xb[i][q] = x[i][q] - dt * uv[i][q];"),
    "edge_velocity_at_the_node": ("orc_velocity_eval(vel, mid, th, ue[i]); /* velocity at the edge centre */",
                                  "orc_velocity_eval(vel, xa, th, ue[i]);"),
    "line_of_the_next_planes": ("    cross3(s[im], s[i], d);\n    double e0[3], e1[3];",
                                "    cross3(s[i], s[(i + 1) % I], d);\n    double e0[3], e1[3];"),
    "velocity_at_the_end_of_step": ("orc_velocity_eval(vel, xa, th, uv[i]);  /* velocity at the vertex */",
                                    "orc_velocity_eval(vel, xa, th + 0.5 * dt, uv[i]);"),
}


@pytest.mark.parametrize("name", sorted(FMFPA_MISTAKES))
def test_fmfpa_pin_catches_planted_mistake(tmp_path, name):
    old, new = FMFPA_MISTAKES[name]
    mut = mutant(tmp_path, old, new, name)
    worst = 0.0
    for gen in ("hex", "tet"):
        m = I.hex_mesh(5) if gen == "hex" else I.kuhn_tet_mesh(3, seed=5)
        om = mut.Mesh(m)
        for vel, ufun, t in ((I.rotation(2 * np.pi), _rot_u, 0.1),
                             (I.deformation(3.0), _deform_u, 0.4)):
            worst = max(worst, _backtrace_residuals(om, m, vel, ufun, t, 0.04))
    assert worst > 1e-6, name


# ------------------------------------------------------------- IDW node values
def _stretched_grid():
    """2 x 2 x 2 cells on the unit cube with the mid plane in x moved from
    0.5 to 0.3: the cells left of it are 0.3 wide, those right of it 0.7."""
    m = dict(I.hex_mesh(2))
    X = m["X"].copy()
    X[np.isclose(X[:, 0], 0.5), 0] = 0.3
    m["X"] = X
    return m


def test_idw_node_value_by_hand(orc):
    """F = 0.2 in the four left cells and 0.8 in the four right ones. The
    centre node (0.3, 0.5, 0.5) is shared by all eight; the left centroids
    (x = 0.15) are at sqrt(0.15^2 + 0.25^2 + 0.25^2) = sqrt(0.1475) from it,
    the right ones (x = 0.65) at sqrt(0.35^2 + 2 * 0.25^2) = sqrt(0.2475).
    Inverse-distance weights (unsquared distances): F* = (0.2 / sqrt(0.1475) + 0.8 /
    sqrt(0.2475)) / (1 / sqrt(0.1475) + 1 / sqrt(0.2475)) = 0.461397...
    (squared distances would give 0.42405..., equal weights 0.5)."""
    m = _stretched_grid()
    om = orc.Mesh(m)
    g = om.geometry()
    F = np.where(g["cell_cen"][:, 0] < 0.3, 0.2, 0.8)
    st = om.taggrid(F)
    v = int(np.argmin(np.abs(m["X"] - np.array([0.3, 0.5, 0.5])).sum(1)))
    a, b = 1.0 / np.sqrt(0.1475), 1.0 / np.sqrt(0.2475)
    hand = (0.2 * a + 0.8 * b) / (a + b)
    assert abs(hand - 0.461397) < 1e-6
    assert abs(st["Fnode"][v] - hand) < 1e-15


IDW_MISTAKES = {
    "squared_distance": ("double w = 1.0 / norm3(d);", "double w = 1.0 / dot3(d, d);"),
    "equal_weights": ("double w = 1.0 / norm3(d);", "double w = 1.0; (void)d;"),
}


@pytest.mark.parametrize("name", sorted(IDW_MISTAKES))
def test_idw_pin_catches_planted_mistake(tmp_path, name):
    old, new = IDW_MISTAKES[name]
    mut = mutant(tmp_path, old, new, name)
    with pytest.raises(AssertionError):
        test_idw_node_value_by_hand(mut)

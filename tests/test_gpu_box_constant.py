"""Plane constants of axis-aligned box cells (Eq. plic-eq on a cuboid).

The mixed path takes a box cell's plane constant from the closed form of the
volume a plane cuts from a cuboid (the root in FP32, relative to the corner
it bounds), one thread per cell after the normals; every other cell, and
every cell of the FP64 path, takes the general method. Whatever the method,
the plane the library returns must cut the cell's fluid fraction from it:
the oracle's FP64 clip of the cell by that plane gives the volume, checked
against F relative to min(F, 1 - F), so that nearly empty and nearly full
cells are held to their own scale.
"""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I
from paper_2111_01524_gb300.partition import cell_centres

pytestmark = pytest.mark.gpu

# relative to min(F, 1 - F): the FP32 root and the FP32 volume function it
# is taken from are good to a few 1e-7 of the volume, FP64 to ~1e-16 of the
# cell
REL_MIXED = 1e-5
REL_FP64 = 1e-8
# of the cell volume: an FP64 plane constant (of the size of the cell) can
# place a plane across a whole face no closer than ~1e-16 of the cell, and
# the oracle's clip rounds at that level too
ABS = 1e-13

EXTREMES = [1e-11, 3e-9, 1e-6, 0.5, 1 - 1e-6, 1 - 3e-9, 1 - 1e-11]


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


def _case(name):
    if name == "aniso":  # sides 1/9 : 0.37/9 : 2.3/9
        m = I.hex_mesh(9, hi=(1.0, 0.37, 2.3))
        body = I.ellipsoid((0.5, 0.18, 1.1), (0.3, 0.12, 0.7))
    elif name == "slab":  # one cell thick: normals in the x-z plane
        n = 30
        m = I.slab_mesh(n)
        x = cell_centres(m)
        r = np.hypot(x[:, 0] - 0.45, x[:, 2] - 0.55)
        F0 = np.clip(0.5 + (0.3 - r) * n, 0.0, 1.0)
    else:
        m = I.hex_mesh(11)
        body = I.sphere((0.4, 0.55, 0.5), 0.3)
    if name != "slab":
        F0 = I.init_fraction(m, body, levels=3)
    # put the extremes on a spread of interfacial cells
    band = np.flatnonzero((F0 > 1e-3) & (F0 < 1 - 1e-3))
    pick = band[:: max(1, band.size // (4 * len(EXTREMES)))]
    F0 = F0.copy()
    F0[pick] = np.resize(EXTREMES, pick.size)
    return m, F0


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["aniso", "slab", "cube"])
def test_box_planes_cut_the_fraction(vof, orc, name, prec):
    m, F0 = _case(name)
    om = orc.Mesh(m)
    ctx = vof.Context(m, precision=vof.PREC_MIXED if prec == "mixed" else vof.PREC_FP64)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    F = ctx.get_fraction()
    P = ctx.planes()
    tc = ctx.tags()[2]
    vol = om.geometry()["cell_vol"]
    band = np.flatnonzero(tc == 0)
    assert band.size > 50
    assert np.isin(EXTREMES, F[band]).sum() == len(EXTREMES)
    rel = REL_MIXED if prec == "mixed" else REL_FP64
    for c in band:
        cut = om.cell_cut_volume(int(c), P[c, :3], P[c, 3]) / vol[c]
        assert abs(cut - F[c]) <= rel * min(F[c], 1.0 - F[c]) + ABS, (int(c), F[c], cut)

"""Parity of the device initialisation (initfgrid, Sec. 3.2) with the oracle,
through the C-ABI: F within 1e-12 for spheres, cylinders and half-spaces on
convex and non-convex cells and several refinements; a batch gives every grid
the body; the state it leaves steps like one set from the host."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS_F64 = 1e-12


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


MESHES = {"hex12": lambda: I.hex_mesh(12), "tet4": lambda: I.kuhn_tet_mesh(4, seed=3),
          "trihex3": lambda: I.trihex_mesh(3, seed=2)}
SHAPES = {"sphere": I.shape_sphere((0.5, 0.52, 0.48), 0.3),
          "cylinder": I.shape_cylinder((0.5, 0.0, 0.55), (0.0, 1.0, 0.0), 0.25),
          "halfspace": I.shape_halfspace((0.5, 0.48, 0.52), (0.3, -0.5, 0.8))}


@pytest.fixture(scope="module")
def meshes(orc):
    return {k: (f(), orc.Mesh(f())) for k, f in MESHES.items()}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("ndiv", [1, 3, 10])
def test_init_fraction_parity(vof, meshes, name, shape, ndiv):
    m, om = meshes[name]
    ctx = vof.Context(m)
    ctx.init_fraction(SHAPES[shape], ndiv)
    F = ctx.get_fraction()
    Fo = om.initfgrid(SHAPES[shape], ndiv)
    assert np.abs(F - Fo).max() < EPS_F64
    assert ((Fo > 0) & (Fo < 1)).sum() > 5


def test_init_fraction_finest_and_mixed_context(vof, meshes):
    m, om = meshes["tet4"]
    Fo = om.initfgrid(SHAPES["sphere"], 16)
    for prec in (vof.PREC_FP64, vof.PREC_MIXED):
        ctx = vof.Context(m, precision=prec)
        ctx.init_fraction(SHAPES["sphere"], 16)
        assert np.abs(ctx.get_fraction() - Fo).max() < EPS_F64


def test_init_fraction_batch(vof, orc):
    grids = [I.hex_mesh(6), I.kuhn_tet_mesh(3, seed=1), I.trihex_mesh(2, seed=3)]
    ctx = vof.Context(grids)
    sh = SHAPES["cylinder"]
    ctx.init_fraction(sh, 6)
    F = ctx.get_fraction()
    Fo = np.concatenate([orc.Mesh(g).initfgrid(sh, 6) for g in grids])
    assert np.abs(F - Fo).max() < EPS_F64


def test_init_fraction_then_step(vof, meshes):
    """A state initialised on the device steps like the same F set from the
    host (the bookkeeping starts from it, the sweeps are full)."""
    m, om = meshes["hex12"]
    vel = I.deformation(3.0)
    a = vof.Context(m)
    a.init_fraction(SHAPES["sphere"], 10)
    b = vof.Context(m)
    b.set_fraction(a.get_fraction())
    for c in (a, b):
        c.reconstruct()
        for k in range(3):
            c.step(vel, 0.01 * k, 0.01)
    assert np.array_equal(a.get_fraction(), b.get_fraction())
    sa, sb = a.stats(), b.stats()
    assert sa["clip_loss"] == sb["clip_loss"] and sa["volume"] == sb["volume"]


def test_init_fraction_rejects_bad_shapes(vof, meshes):
    m, _ = meshes["hex12"]
    ctx = vof.Context(m)
    bad = [I.Shape(9, (0.5, 0.5, 0.5), r=0.1), I.Shape(I.Shape.SPHERE, (0.5, 0.5, 0.5), r=0.0),
           I.Shape(I.Shape.CYLINDER, (0.5, 0.5, 0.5), (0, 0, 1), r=-1.0)]
    for sh in bad:
        with pytest.raises(vof.VofError) as e:
            ctx.init_fraction(sh, 10)
        assert e.value.status == vof.VOF_EINVAL
    for ndiv in (0, 17):
        with pytest.raises(vof.VofError):
            ctx.init_fraction(SHAPES["sphere"], ndiv)
    sh = SHAPES["halfspace"]
    s = vof.shape_struct(sh)
    s.a[0] *= 2.0  # not a unit vector
    import ctypes
    assert vof.lib().vof_init_fraction(ctx._h, ctypes.byref(s), 10, None) == vof.VOF_EINVAL

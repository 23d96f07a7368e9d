"""Quasi-2D grids (one cell across y) and the 2D deformation test (Sec. 4.3)
through the C-ABI against the oracle: the singular LSGIR system solved by its
pseudo-inverse, one step and coupled steps of the x-z field, the device
initialisation of the cylinder, and no flux through the y-faces."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS_F64 = 1e-12
EPS_MIXED = 1e-6
CYL = I.shape_cylinder((0.5, 0.0, 0.75), (0.0, 1.0, 0.0), 0.15)


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


@pytest.fixture(scope="module")
def slab(orc):
    m = I.slab_mesh(24)
    om = orc.Mesh(m)
    return m, om, om.initfgrid(CYL, 10)


def test_quasi2d_lsgir_planes(vof, slab):
    m, om, F0 = slab
    x = om.geometry()["cell_cen"]
    for F in (F0, np.clip(0.5 + (x - 0.5) @ [0.8, 0.3, -0.6], 0.0, 1.0)):
        ctx = vof.Context(m, precision=vof.PREC_FP64)
        ctx.set_fraction(F)
        ctx.reconstruct()
        st = om.reconstruct(F)
        band = st["tag_c"] == 0
        P = ctx.planes()
        assert band.sum() > 20
        assert np.abs(P[band, :3] - st["nrm"][band]).max() < EPS_F64
        assert np.abs(P[band, 1]).max() < 1e-12  # in-plane normals
        h = np.sqrt(om.geometry()["cell_vol"])
        assert (np.abs(P[band, 3] - st["C"][band]) / h[band]).max() < EPS_F64


def test_quasi2d_device_init(vof, slab):
    m, om, F0 = slab
    ctx = vof.Context(m)
    ctx.init_fraction(CYL, 10)
    assert np.abs(ctx.get_fraction() - F0).max() < EPS_F64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_quasi2d_one_step(vof, slab, prec):
    m, om, F0 = slab
    vel = I.deformation2d(8.0)
    p = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    ctx = vof.Context(m, precision=p)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    dt = om.suggest_dt(vel, 0.0, 0.5, 8.0)
    assert abs(ctx.suggest_dt(vel, 0.0, 0.5, 8.0) - dt) <= 1e-14 * dt
    ctx.advect(vel, 0.0, dt)
    Vd, VF = ctx.face_flux()
    Vdo, VFo, _ = om.faceflux(vel, 0.0, dt, st)
    Fo = om.vofadv(st["F"], Vdo, VFo)
    V = om.geometry()["cell_vol"]
    ny = np.abs(om.geometry()["face_nrm"][:, 1]) > 0.5
    assert np.all(Vd[ny] == 0.0) and np.all(VF[ny] == 0.0)
    tol = EPS_F64 if prec == "fp64" else EPS_MIXED
    assert np.abs(ctx.get_fraction() - Fo).max() < tol
    assert (np.abs(VF - VFo) / V[m["owner"]]).max() < tol
    assert ctx.stats()["n_overflow"] == 0


def test_quasi2d_coupled_steps(vof, orc):
    """32 x 1 x 32, 12 coupled steps of the 2D deformation test at CFL 0.5:
    each side runs the loop on its own; F within 1e-12 after every step."""
    m = I.slab_mesh(32)
    om = orc.Mesh(m)
    F0 = om.initfgrid(CYL, 10)
    vel = I.deformation2d(8.0)
    ctx = vof.Context(m, precision=vof.PREC_FP64)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    t = 0.0
    for k in range(12):
        dt = om.suggest_dt(vel, t, 0.5, 8.0)
        ctx.step(vel, t, dt)
        st = om.step(vel, t, dt, st)
        t += dt
        assert np.abs(ctx.get_fraction() - st["F"]).max() < EPS_F64, k
    s = ctx.stats()
    V = om.geometry()["cell_vol"]
    vol0 = float((V * F0).sum())
    resid = s["volume"] - (vol0 - s["clip_loss"] - s["cutoff_loss"] - s["boundary_outflow"])
    assert abs(resid) < 1e-12 * vol0

"""Parity of the LSFIR reconstruction (Sec. 2.1.2) of the CUDA library with
the FP64 oracle, through the C-ABI.

Bars: FP64 planes within 1e-12 (normals; plane constants relative to the
cell size) and F within 1e-12 after advection; mixed F within 1e-6; the
LSGIR path (the default) unchanged.
"""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS_F64 = 1e-12
EPS_MIXED = 1e-6


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


def _case(name):
    if name == "hex12":
        return I.hex_mesh(12), I.sphere((0.35, 0.35, 0.35), 0.15)
    if name == "hex7":  # ragged: no size is a multiple of a block or warp
        return I.hex_mesh(7), I.sphere((0.45, 0.5, 0.52), 0.3)
    if name == "tet5":
        return I.kuhn_tet_mesh(5, seed=3), I.sphere((0.5, 0.55, 0.5), 0.3)
    if name == "trihex3":  # non-convex cells
        return I.trihex_mesh(3, seed=2), I.sphere((0.5, 0.48, 0.52), 0.3)
    if name == "hex32":
        return I.hex_mesh(32), I.sphere((0.35, 0.35, 0.35), 0.15)
    raise KeyError(name)


CASES = ["hex12", "hex7", "tet5", "trihex3"]


@pytest.fixture(scope="module")
def cases(orc):
    out = {}
    for n in CASES + ["hex32"]:
        m, body = _case(n)
        out[n] = (m, I.init_fraction(m, body, levels=3), orc.Mesh(m))
    return out


@pytest.mark.parametrize("name", CASES)
def test_lsfir_planes_parity_fp64(vof, orc, cases, name):
    m, F0, om = cases[name]
    ctx = vof.Context(m, precision=vof.PREC_FP64, recon=vof.RECON_LSFIR)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0, recon=orc.LSFIR)
    tv, tf, tc = ctx.tags()
    assert np.array_equal(tc, st["tag_c"])
    P = ctx.planes()
    band = st["tag_c"] == 0
    h = np.cbrt(om.geometry()["cell_vol"])
    assert np.abs(P[band, :3] - st["nrm"][band]).max() < EPS_F64
    assert (np.abs(P[band, 3] - st["C"][band]) / h[band]).max() < EPS_F64
    # LSFIR moved the normals away from LSGIR's
    ref = vof.Context(m, precision=vof.PREC_FP64)
    ref.set_fraction(F0)
    ref.reconstruct()
    assert np.abs(ref.planes()[band, :3] - P[band, :3]).max() > 1e-3


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lsfir_advect_parity(vof, orc, cases, name, prec):
    m, F0, om = cases[name]
    vel = I.deformation(3.0)
    p = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    ctx = vof.Context(m, precision=p, recon=vof.RECON_LSFIR)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0, recon=orc.LSFIR)
    dt = om.suggest_dt(vel, 0.0, 0.5, 1e9)
    ctx.advect(vel, 0.0, dt)
    Vd, VF = ctx.face_flux()
    Vdo, VFo, _ = om.faceflux(vel, 0.0, dt, st)
    Fo = om.vofadv(st["F"], Vdo, VFo)
    V = om.geometry()["cell_vol"]
    if prec == "fp64":
        assert np.abs(VF - VFo).max() < EPS_F64 * V.min()
        assert np.abs(ctx.get_fraction() - Fo).max() < EPS_F64
    else:
        assert np.abs(ctx.get_fraction() - Fo).max() < EPS_MIXED
        assert (np.abs(VF - VFo) / V[m["owner"]]).max() < EPS_MIXED
    assert ctx.stats()["n_overflow"] == 0


def test_lsfir_multistep_parity_hex32_deformation(vof, orc, cases):
    """32^3 deformation, 6 coupled steps at CFL 0.5 with LSFIR: each side
    runs the loop on its own; F within 1e-12 after every step. The planes
    after the last step are compared at 1e-10: each side reconstructs its own
    F, and the least-squares fit of neighbouring centres amplifies the
    rounding-level differences of F (from the same F they agree to 1e-12,
    test_lsfir_planes_parity_fp64)."""
    m, F0, om = cases["hex32"]
    vel = I.deformation(3.0)
    ctx = vof.Context(m, precision=vof.PREC_FP64, recon=vof.RECON_LSFIR)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0, recon=orc.LSFIR)
    t = 0.0
    for k in range(6):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        ctx.step(vel, t, dt)
        st = om.step(vel, t, dt, st, recon=orc.LSFIR)
        t += dt
        assert np.abs(ctx.get_fraction() - st["F"]).max() < EPS_F64, k
    P = ctx.planes()
    band = st["tag_c"] == 0
    assert np.abs(P[band, :3] - st["nrm"][band]).max() < 1e-10


def test_lsfir_iteration_limits(vof, orc, cases):
    """Other iteration limits and tolerances give the oracle's planes for
    the same settings (one iteration; stop after the first; eight)."""
    m, F0, om = cases["tet5"]
    for n_out, tol in ((1, 1e-3), (2, 0.5), (8, 1e-6)):
        ctx = vof.Context(m, precision=vof.PREC_FP64, recon=vof.RECON_LSFIR,
                          lsfir_max_iter=n_out, lsfir_tol=tol)
        ctx.set_fraction(F0)
        ctx.reconstruct()
        st = om.taggrid(F0)
        ng = om.lsgir(st["F"], st["tag_c"])
        nrm, C, it = om.lsfir(st["F"], st["tag_c"], ng, n_out=n_out, tol=tol)
        band = st["tag_c"] == 0
        P = ctx.planes()
        assert np.abs(P[band, :3] - nrm[band]).max() < EPS_F64, (n_out, tol, it)


def test_lsfir_graph_replay_matches_launches(vof, cases):
    """A captured step with the LSFIR reconstruction (fixed launch sequence,
    converged iterations skip their work on the device) replays the
    launched steps bit for bit."""
    import torch
    m, F0, om = cases["tet5"]
    vel = I.rotation(2 * np.pi)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = vof.Context(m, precision=vof.PREC_MIXED, recon=vof.RECON_LSFIR)
        b = vof.Context(m, precision=vof.PREC_MIXED, recon=vof.RECON_LSFIR)
        for c in (a, b):
            c.set_fraction(F0)
            c.reconstruct()
        a.graph_capture(with_reconstruct=True)
        t = np.zeros(1)
        for _ in range(4):
            dt = a.suggest_dt_batch([vel], t, 0.5, np.full(1, 10.0))
            a.graph_launch([vel], t, dt)
            b.step_batch([vel], t, dt)
            t = t + dt
        Fa, Fb = a.get_fraction(), b.get_fraction()
        Pa, Pb = a.planes(), b.planes()
    assert np.array_equal(Fa, Fb) and np.array_equal(Pa, Pb)
    assert not np.array_equal(Fa, F0)

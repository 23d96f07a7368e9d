"""Parity of the EMFPA path (edge-matched flux polyhedra, Sec. 2.2.1) of the
CUDA library with the FP64 oracle, through the C-ABI.

Same bars as the FMFPA path: polyhedra within 1e-13 (FP64); FP64 F within
1e-12 absolute and V_F within 1e-12 V_cell; mixed F within 1e-6 and V_F
within 1e-6 V_owner; exact shift at CFL 1; no capacity overflow.
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
    if name == "tet4":
        return I.kuhn_tet_mesh(4, seed=3), I.sphere((0.5, 0.55, 0.5), 0.27)
    if name == "trihex3":  # non-convex cells
        return I.trihex_mesh(3, seed=2), I.sphere((0.5, 0.48, 0.52), 0.3)
    if name == "hex32":
        return I.hex_mesh(32), I.sphere((0.35, 0.35, 0.35), 0.15)
    raise KeyError(name)


CASES = ["hex12", "hex7", "tet4", "trihex3"]


@pytest.fixture(scope="module")
def cases(orc):
    out = {}
    for n in CASES + ["hex32"]:
        m, body = _case(n)
        out[n] = (m, I.init_fraction(m, body, levels=3), orc.Mesh(m))
    return out


VELS = {"deformation": I.deformation(3.0), "rotation": I.rotation(2 * np.pi),
        "translation": I.translation((0.7, -0.4, 0.25))}


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_emfpa_polyhedra_parity(vof, cases, name, prec):
    m, F0, om = cases[name]
    p = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    ctx = vof.Context(m, precision=p, flux=vof.FLUX_EMFPA)
    vel = VELS["deformation"]
    dt = om.suggest_dt(vel, 0.2, 0.5, 3.0)
    faces = np.arange(0, om.n_face, 2, dtype=np.int32)
    got = ctx.flux_polyhedra(vel, 0.2, dt, faces)
    A = om.geometry()["face_area"]
    worst = 0.0
    for f, P in zip(faces, got):
        Po, vd, fl = om.emfpa(int(f), vel, 0.2 + 0.5 * dt, dt)
        assert P is not None and P.shape == Po.shape, f
        if fl & 2:
            continue  # edge-on back-traced loop: apex placement undefined
        worst = max(worst, np.abs(P - Po).max() / np.sqrt(A[f]))
    # FP64: rounding; mixed: FP32 in face-local units of sqrt(A)
    assert worst < (1e-13 if prec == "fp64" else 1e-5), worst


def _one_step(vof, m, F0, om, vel, precision, t=0.0, cfl=0.5):
    ctx = vof.Context(m, precision=precision, flux=vof.FLUX_EMFPA)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    dt = om.suggest_dt(vel, t, cfl, 1e9)
    ctx.advect(vel, t, dt)
    Vd, VF = ctx.face_flux()
    Vdo, VFo, stats = om.faceflux(vel, t, dt, st, method=1)
    return ctx, st, (Vd, VF, ctx.get_fraction()), (Vdo, VFo, om.vofadv(st["F"], Vdo, VFo))


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("vname", sorted(VELS))
def test_emfpa_advect_parity_fp64(vof, cases, name, vname):
    m, F0, om = cases[name]
    ctx, st, (Vd, VF, F), (Vdo, VFo, Fo) = _one_step(vof, m, F0, om, VELS[vname], vof.PREC_FP64)
    V = om.geometry()["cell_vol"]
    assert np.abs(Vd - Vdo).max() <= 1e-14 * np.abs(Vdo).max() + 1e-30
    assert np.abs(VF - VFo).max() < EPS_F64 * V.min()
    assert np.abs(F - Fo).max() < EPS_F64
    s = ctx.stats()
    assert s["n_overflow"] == 0
    assert s["n_degenerate"] == 0  # every vertex uses its own streak line
    assert s["n_active_faces"] == int((st["tag_f"] == 0).sum())


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("vname", ["deformation", "rotation"])
def test_emfpa_advect_parity_mixed(vof, cases, name, vname):
    m, F0, om = cases[name]
    ctx, st, (Vd, VF, F), (Vdo, VFo, Fo) = _one_step(vof, m, F0, om, VELS[vname], vof.PREC_MIXED)
    V = om.geometry()["cell_vol"]
    assert np.abs(F - Fo).max() < EPS_MIXED
    assert (np.abs(VF - VFo) / V[m["owner"]]).max() < EPS_MIXED
    assert ctx.stats()["n_overflow"] == 0


def test_emfpa_multistep_parity_hex32_deformation(vof, cases):
    """32^3 deformation, 10 coupled steps at CFL 0.5 with EMFPA: the GPU and
    the oracle each run the loop on their own; F agrees to 1e-12 after every
    step and the volume bookkeeping closes."""
    m, F0, om = cases["hex32"]
    vel = I.deformation(3.0)
    ctx = vof.Context(m, precision=vof.PREC_FP64, flux=vof.FLUX_EMFPA)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    t = 0.0
    V = om.geometry()["cell_vol"]
    vol0 = float((V * st["F"]).sum())
    for k in range(10):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        ctx.step(vel, t, dt)
        st = om.step(vel, t, dt, st, method=1)
        t += dt
        assert np.abs(ctx.get_fraction() - st["F"]).max() < EPS_F64, k
    s = ctx.stats()
    resid = s["volume"] - (vol0 - s["clip_loss"] - s["cutoff_loss"] - s["boundary_outflow"])
    assert abs(resid) < 1e-12 * vol0
    assert s["n_overflow"] == 0


def test_emfpa_cfl1_translation_exact_shift_gpu(vof):
    n = 8
    m = I.hex_mesh(n)
    F0 = I.init_fraction(m, I.sphere((0.45, 0.52, 0.48), 0.3), levels=3)
    ctx = vof.Context(m, precision=vof.PREC_FP64, flux=vof.FLUX_EMFPA)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    F = ctx.get_fraction().reshape(n, n, n)
    ctx.advect(I.translation((1.0, 0.0, 0.0)), 0.0, 1.0 / n)
    G = ctx.get_fraction().reshape(n, n, n)
    assert np.abs(G[:, :, 1:] - F[:, :, :-1]).max() < 4e-15
    assert np.abs(G[:, :, 0]).max() == 0.0


def test_emfpa_and_fmfpa_agree_for_uniform_flow_gpu(vof, cases):
    """Uniform flow: both constructions give the exact prism, so the two
    library paths give the same face volumes up to rounding."""
    m, F0, om = cases["tet4"]
    vel = VELS["translation"]
    out = []
    for flux in (vof.FLUX_FMFPA, vof.FLUX_EMFPA):
        ctx = vof.Context(m, precision=vof.PREC_FP64, flux=flux)
        ctx.set_fraction(F0)
        ctx.reconstruct()
        ctx.advect(vel, 0.0, om.suggest_dt(vel, 0.0, 0.6, 1e9))
        out.append(ctx.face_flux()[1])
    V = om.geometry()["cell_vol"]
    assert np.abs(out[1] - out[0]).max() < EPS_F64 * V.min()

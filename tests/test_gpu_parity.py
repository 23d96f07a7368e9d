"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances: connectivity, candidate lists and tags bit-exact; FP64 path F
within 1e-12 absolute, per-face volumes within 1e-12 of the cell volume;
mixed path F within 1e-6 absolute.
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
        m = I.hex_mesh(12)
        body = I.sphere((0.35, 0.35, 0.35), 0.15)
    elif name == "hex7":  # ragged: no size is a multiple of a block or warp
        m = I.hex_mesh(7)
        body = I.sphere((0.45, 0.5, 0.52), 0.3)
    elif name == "tet4":
        m = I.kuhn_tet_mesh(4, seed=3)
        body = I.sphere((0.5, 0.55, 0.5), 0.27)
    elif name == "trihex3":  # distorted cubic cells, triangulated faces, non-convex
        m = I.trihex_mesh(3, seed=2)
        body = I.sphere((0.5, 0.48, 0.52), 0.3)
    elif name == "hex32":
        m = I.hex_mesh(32)
        body = I.sphere((0.35, 0.35, 0.35), 0.15)
    else:
        raise KeyError(name)
    F0 = I.init_fraction(m, body, levels=3)
    return m, F0


CASES = ["hex12", "hex7", "tet4", "trihex3"]


@pytest.fixture(scope="module")
def cases(orc):
    out = {}
    for n in CASES + ["hex32"]:
        m, F0 = _case(n)
        out[n] = (m, F0, orc.Mesh(m))
    return out


@pytest.mark.parametrize("name", CASES)
def test_geometry_parity(vof, cases, name):
    m, F0, om = cases[name]
    ctx = vof.Context(m)
    g, go = ctx.geometry(), om.geometry()
    assert np.allclose(g["cell_vol"], go["cell_vol"], rtol=1e-14, atol=0)
    for k in ("cell_cen", "face_cen", "face_nrm"):
        assert np.abs(g[k] - go[k]).max() < 1e-15, k
    assert np.allclose(g["face_area"], go["face_area"], rtol=1e-14, atol=0)


@pytest.mark.parametrize("name", CASES)
def test_connectivity_bit_exact(vof, cases, name):
    m, F0, om = cases[name]
    ctx = vof.Context(m)
    p, i = ctx.neighbors()
    po, io = om.neighbors()
    assert np.array_equal(p, po) and np.array_equal(i, io)
    faces = np.arange(om.n_face, dtype=np.int32)
    got = ctx.candidates(faces)
    for f in faces:
        assert np.array_equal(got[f], om.candidates(f)), f


@pytest.mark.parametrize("name", CASES)
def test_reconstruct_parity_fp64(vof, cases, name):
    m, F0, om = cases[name]
    ctx = vof.Context(m, precision=vof.PREC_FP64)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    tv, tf, tc = ctx.tags()
    assert np.array_equal(tc, st["tag_c"])
    assert np.array_equal(tv, st["tag_v"])
    assert np.array_equal(ctx.get_fraction(), st["F"])  # cut-off is exact
    P = ctx.planes()
    band = st["tag_c"] == 0
    assert band.sum() > 10
    h = np.cbrt(om.geometry()["cell_vol"])
    assert np.abs(P[band, :3] - st["nrm"][band]).max() < 1e-12
    assert (np.abs(P[band, 3] - st["C"][band]) / h[band]).max() < 1e-12
    assert np.all(P[~band] == 0)


@pytest.mark.parametrize("name", ["hex12", "tet4"])
def test_flux_polyhedra_parity(vof, cases, name):
    m, F0, om = cases[name]
    ctx = vof.Context(m)
    vel = I.deformation(3.0)
    dt = om.suggest_dt(vel, 0.2, 0.5, 3.0)
    faces = np.arange(0, om.n_face, 3, dtype=np.int32)
    got = ctx.flux_polyhedra(vel, 0.2, dt, faces)
    for f, P in zip(faces, got):
        Po, vd, fl = om.fmfpa(int(f), vel, 0.2 + 0.5 * dt, dt)
        assert P.shape == Po.shape
        if fl & 2:
            continue  # edge-on loop: apex placement is undefined
        assert np.abs(P - Po).max() < 1e-13, f


def _one_step(vof, m, F0, om, vel, precision, t=0.0, cfl=0.5):
    ctx = vof.Context(m, precision=precision)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    dt = om.suggest_dt(vel, t, cfl, 1e9)
    assert abs(ctx.suggest_dt(vel, t, cfl, 1e9) - dt) <= 1e-14 * dt
    ctx.advect(vel, t, dt)
    Vd, VF = ctx.face_flux()
    Vdo, VFo, stats = om.faceflux(vel, t, dt, st)
    Fadv = ctx.get_fraction()
    Fo = om.vofadv(st["F"], Vdo, VFo)
    return ctx, st, (Vd, VF, Fadv), (Vdo, VFo, Fo)


VELS = {"deformation": I.deformation(3.0), "rotation": I.rotation(2 * np.pi),
        "translation": I.translation((0.7, -0.4, 0.25))}


def _cfl(name):
    """CFL of the one-step cases: 0.4 on the jittered tetrahedra (as their rotation workload),
    where the candidate ring covers every interior flux polyhedron; at 0.5
    the diagonal translation already carries a few polyhedra of the 4^3 x 6
    grid past it (the CFL bound measures cells by their bounding boxes)."""
    return 0.4 if name.startswith("tet") else 0.5


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("vname", sorted(VELS))
def test_advect_parity_fp64(vof, cases, name, vname):
    m, F0, om = cases[name]
    vel = VELS[vname]
    ctx, st, (Vd, VF, F), (Vdo, VFo, Fo) = _one_step(vof, m, F0, om, vel, vof.PREC_FP64,
                                                     cfl=_cfl(name))
    V = om.geometry()["cell_vol"]
    assert np.abs(Vd - Vdo).max() <= 1e-14 * np.abs(Vdo).max() + 1e-30
    assert np.abs(VF - VFo).max() < EPS_F64 * V.min()
    assert np.abs(F - Fo).max() < EPS_F64
    tv, tf, tc = ctx.tags()
    assert np.array_equal(tf, st["tag_f"])
    s = ctx.stats()
    assert s["n_overflow"] == 0
    assert s["n_active_faces"] == int((st["tag_f"] == 0).sum())


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("vname", sorted(VELS))
def test_advect_parity_mixed(vof, cases, name, vname):
    m, F0, om = cases[name]
    vel = VELS[vname]
    ctx, st, (Vd, VF, F), (Vdo, VFo, Fo) = _one_step(vof, m, F0, om, vel, vof.PREC_MIXED,
                                                     cfl=_cfl(name))
    V = om.geometry()["cell_vol"]
    assert np.abs(F - Fo).max() < EPS_MIXED
    # a face volume error moves F of its owner by dVF / V_owner
    assert (np.abs(VF - VFo) / V[m["owner"]]).max() < EPS_MIXED
    s = ctx.stats()
    assert s["n_overflow"] == 0 and s["n_escaped"] == 0


@pytest.mark.parametrize("name", CASES)
def test_multistep_tags_and_band_sweeps(vof, cases, name):
    """After the first step the sweeps are band-limited (only the cells, nodes
    and faces the step can change are visited): over 8 coupled steps the node
    and cell tags equal the oracle's full sweeps bit for bit, the face tags
    each advect uses equal the oracle's of the state it advects, and F stays
    within 1e-12."""
    m, F0, om = cases[name]
    vel = VELS["rotation"] if name.startswith("tet") else VELS["deformation"]
    ctx = vof.Context(m, precision=vof.PREC_FP64)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    t = 0.0
    for k in range(8):
        dt = om.suggest_dt(vel, t, 0.5, 10.0)
        prev = st
        ctx.step(vel, t, dt)
        st = om.step(vel, t, dt, st)
        t += dt
        tv, tf, tc = ctx.tags()
        assert np.array_equal(tv, st["tag_v"]), (name, k)
        assert np.array_equal(tc, st["tag_c"]), (name, k)
        assert np.array_equal(tf, prev["tag_f"]), (name, k)
        assert np.abs(ctx.get_fraction() - st["F"]).max() < EPS_F64, (name, k)
    assert ctx.stats()["n_interfacial"] == int((st["tag_c"] == 0).sum())


def test_multistep_parity_hex32_deformation(vof, cases):
    """32^3 deformation, 10 steps at CFL 0.5: the GPU and the oracle each
    run the whole loop on their own; F agrees to 1e-12 after every step."""
    m, F0, om = cases["hex32"]
    vel = I.deformation(3.0)
    ctx = vof.Context(m, precision=vof.PREC_FP64)
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    t = 0.0
    V = om.geometry()["cell_vol"]
    vol0 = (V * st["F"]).sum()
    for k in range(10):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        ctx.step(vel, t, dt)
        st = om.step(vel, t, dt, st)
        t += dt
        F = ctx.get_fraction()
        assert np.abs(F - st["F"]).max() < EPS_F64, k
    s = ctx.stats()
    assert abs(s["volume"] - vol0) < 1e-12 * vol0
    assert s["n_overflow"] == 0


def test_full_cycle_hex32_deformation(vof, cases):
    """32^3 deformation over the whole cycle (t = 0 -> T = 3, 250 steps at
    CFL 0.5): the FP64 path stays within 1e-12 of the oracle at every step
    although each side feeds back its own results; the mixed path's shape
    error E_shape = sum V |F(T) - F(0)| (Sec. 4.2) agrees with the oracle's to
    1e-5 relative and both conserve volume to 1e-12 in the bookkeeping."""
    m, F0, om = cases["hex32"]
    vel = I.deformation(3.0)
    c64 = vof.Context(m, precision=vof.PREC_FP64)
    cmx = vof.Context(m, precision=vof.PREC_MIXED)
    for c in (c64, cmx):
        c.set_fraction(F0)
        c.reconstruct()
    st = om.reconstruct(F0)
    V = om.geometry()["cell_vol"]
    vol0 = float((V * F0).sum())
    t, k = 0.0, 0
    while t < 3.0 - 1e-14:
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        assert dt == c64.suggest_dt(vel, t, 0.5, 3.0)
        st = om.step(vel, t, dt, st)
        c64.step(vel, t, dt)
        cmx.step(vel, t, dt)
        t += dt
        k += 1
        if k % 10 == 0:
            assert np.abs(c64.get_fraction() - st["F"]).max() < EPS_F64, k
    assert k == 250
    Fo, F64, Fm = st["F"], c64.get_fraction(), cmx.get_fraction()
    assert np.abs(F64 - Fo).max() < EPS_F64
    es_o = float((V * np.abs(Fo - F0)).sum())
    es_m = float((V * np.abs(Fm - F0)).sum())
    assert abs(es_m - es_o) < 1e-5 * es_o, (es_m, es_o)
    for c in (c64, cmx):
        s = c.stats()
        resid = s["volume"] - (vol0 - s["clip_loss"] - s["cutoff_loss"] - s["boundary_outflow"])
        assert abs(resid) < 1e-12 * vol0


def test_cfl1_translation_exact_shift_gpu(vof):
    n = 8
    m = I.hex_mesh(n)
    F0 = I.init_fraction(m, I.sphere((0.45, 0.52, 0.48), 0.3), levels=3)
    for prec in (vof.PREC_FP64,):
        ctx = vof.Context(m, precision=prec)
        ctx.set_fraction(F0)
        ctx.reconstruct()
        F = ctx.get_fraction().reshape(n, n, n)
        ctx.advect(I.translation((1.0, 0.0, 0.0)), 0.0, 1.0 / n)
        G = ctx.get_fraction().reshape(n, n, n)
        assert np.abs(G[:, :, 1:] - F[:, :, :-1]).max() < 4e-15
        assert np.abs(G[:, :, 0]).max() == 0.0


def test_edge_cases(vof):
    m = I.hex_mesh(5)
    vel = I.deformation(3.0)
    for value in (0.0, 1.0):
        ctx = vof.Context(m)
        ctx.set_fraction(np.full(125, value))
        ctx.reconstruct()
        ctx.step(vel, 0.0, 0.02)
        s = ctx.stats()
        assert s["n_active_faces"] == 0 and s["n_interfacial"] == 0
        assert np.all(ctx.get_fraction() == value)
    # a single interfacial cell in an empty grid
    F = np.zeros(125)
    F[62] = 0.3
    ctx = vof.Context(m)
    ctx.set_fraction(F)
    ctx.reconstruct()
    ctx.step(I.translation((0.3, 0.2, -0.1)), 0.0, 0.05)
    G = ctx.get_fraction()
    V = ctx.geometry()["cell_vol"]
    assert abs((V * G).sum() - 0.3 * V[62]) < 1e-17
    assert G.min() >= 0 and G.max() <= 1


def test_invalid_inputs_are_rejected(vof):
    ctx = vof.Context(I.hex_mesh(3))
    ctx.set_fraction(np.full(27, 0.5))
    with pytest.raises(vof.VofError) as e:
        ctx.advect(I.deformation(3.0), 0.0, 0.01)  # needs a reconstruction
    assert e.value.status == vof.VOF_ESTATE
    with pytest.raises(vof.VofError):
        ctx.candidates([10 ** 6])
    bad = dict(I.hex_mesh(2))
    bad["owner"] = bad["owner"].copy()
    bad["owner"][0] = 99
    with pytest.raises(vof.VofError) as e:
        vof.Context(bad)
    assert e.value.status == vof.VOF_EINVAL
    bad = dict(I.hex_mesh(2))
    bad["neighbour"] = bad["neighbour"].copy()
    inner = int(np.nonzero(bad["neighbour"] >= 0)[0][0])
    bad["neighbour"][inner] = bad["owner"][inner]
    with pytest.raises(vof.VofError):
        vof.Context(bad)


@pytest.mark.parametrize("flux", ["FMFPA", "EMFPA", "NMFPA"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_planar_interface_translates_exactly_gpu(vof, flux, prec):
    """A planar interface x = 0.43 with exact cell fractions in the uniform
    flow u = (1, 0, 0) at CFL 0.3: PLIC holds the plane exactly and every
    construction is the exact prism of the face, so one step gives the exact
    fractions of the plane at x = 0.43 + dt (FP64 to rounding, mixed within
    its FP32 geometry). Cells next to the inflow wall are left out."""
    n = 8
    h = 1.0 / n
    m = I.hex_mesh(n)
    ctx = vof.Context(m, precision=vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED,
                      flux=getattr(vof, "FLUX_" + flux))
    x = ctx.geometry()["cell_cen"][:, 0]
    ctx.set_fraction(np.clip((0.43 - (x - 0.5 * h)) / h, 0.0, 1.0))
    ctx.reconstruct()
    dt = 0.3 * h
    ctx.advect(I.translation((1.0, 0.0, 0.0)), 0.0, dt)
    exact = np.clip((0.43 + dt - (x - 0.5 * h)) / h, 0.0, 1.0)
    keep = x > 1.5 * h
    err = np.abs(ctx.get_fraction()[keep] - exact[keep]).max()
    assert err < (1e-13 if prec == "fp64" else EPS_MIXED), err
    assert ctx.stats()["n_overflow"] == 0


def _boundary_case(kind):
    """A body on each side of the domain in a uniform flow with inflow and
    outflow walls: one across x = 1 (fluid leaves), one across x = 0 and
    y = 0 (the flow enters there and carries no fluid from outside)."""
    if kind == "hex":
        m = I.hex_mesh(10)
    else:
        m = I.kuhn_tet_mesh(4, seed=3)
    Fa = I.init_fraction(m, I.sphere((0.93, 0.55, 0.5), 0.22), levels=3)
    Fb = I.init_fraction(m, I.sphere((0.04, 0.06, 0.45), 0.25), levels=3)
    return m, np.minimum(1.0, Fa + Fb), I.translation((0.8, 0.35, -0.25))


@pytest.mark.parametrize("kind", ["hex", "tet"])
@pytest.mark.parametrize("flux", ["FMFPA", "EMFPA", "NMFPA"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_boundary_crossing_parity(vof, orc, kind, flux, prec):
    """Faces on the domain boundary and interior faces whose polyhedra reach
    outside it (no fluid outside the domain), element by element against the
    oracle: V_F of every face and F after one step, and F after 4 coupled
    steps, for the three constructions."""
    m, F0, vel = _boundary_case(kind)
    om = orc.Mesh(m)
    method = getattr(orc, flux)
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    tol = EPS_F64 if prec == "fp64" else EPS_MIXED
    ctx = vof.Context(m, precision=P, flux=getattr(vof, "FLUX_" + flux))
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = om.reconstruct(F0)
    V = om.geometry()["cell_vol"]
    bnd = m["neighbour"] < 0
    t = 0.0
    for k in range(4):
        dt = om.suggest_dt(vel, t, 0.5, 10.0)
        ctx.advect(vel, t, dt)
        Vd, VF = ctx.face_flux()
        Vdo, VFo, _ = om.faceflux(vel, t, dt, st, method=method)
        if k == 0:
            act = st["tag_f"] == 0
            assert (act & bnd).sum() > 10  # boundary faces with geometric fluxes
            assert (VFo[bnd] > 0).any() and (Vdo[bnd] < 0).any()  # outflow and inflow
        err = np.abs(VF - VFo) / V[m["owner"]]
        assert err.max() < tol, (k, int(err.argmax()), bool(bnd[err.argmax()]))
        ctx.reconstruct()
        st = om.step(vel, t, dt, st, method=method)
        t += dt
        assert np.abs(ctx.get_fraction() - st["F"]).max() < tol * (1 if prec == "fp64" else 4), k
    s = ctx.stats()
    assert s["n_overflow"] == 0 and s["n_escaped"] == 0
    assert s["boundary_outflow"] > 0


@pytest.mark.parametrize("flux", ["FMFPA", "EMFPA"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_in_kernel_construction_fallback(vof, cases, flux, prec):
    """Active faces beyond the prebuilt-polyhedron capacity are built inside
    the flux kernel by one lane with the same arithmetic: a context whose
    capacity is 5 faces gives the same F, tags and face volumes bit for bit
    as one with room for all, over 3 coupled steps (FP64: and the oracle's F
    to 1e-12)."""
    m, F0, om = cases["hex12"]
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    kw = dict(precision=P, flux=getattr(vof, "FLUX_" + flux))
    full = vof.Context(m, **kw)
    small = vof.Context(m, poly_capacity=5, **kw)
    vel = VELS["deformation"]
    st = om.reconstruct(F0)
    for c in (full, small):
        c.set_fraction(F0)
        c.reconstruct()
    t = 0.0
    for _ in range(3):
        dt = om.suggest_dt(vel, t, 0.5, 3.0)
        full.step(vel, t, dt)
        small.step(vel, t, dt)
        st = om.step(vel, t, dt, st, method=getattr(orc_methods(), flux))
        t += dt
        assert np.array_equal(full.face_flux()[1], small.face_flux()[1])
        assert np.array_equal(full.get_fraction(), small.get_fraction())
        assert small.stats()["n_active_faces"] > 100
    if prec == "fp64":
        assert np.abs(small.get_fraction() - st["F"]).max() < EPS_F64
    with pytest.raises(vof.VofError) as e:
        vof.Context(m, poly_capacity=-1)
    assert e.value.status == vof.VOF_EINVAL


def orc_methods():
    import oracle
    return oracle

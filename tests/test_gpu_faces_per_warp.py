"""Two faces per warp: the flux kernel with one flux polyhedron per half
warp (16 lanes) gives the same face volumes and F as one per warp, bit for
bit (every reduction keeps its order: a whole warp whose upper lanes hold 0
sums as a half warp does), for FMFPA on tetrahedra and NMFPA on hexahedra
and tetrahedra, both precisions, over coupled steps, with no loop list
overflowing; it is refused where the polyhedron's faces plus a cell's faces
plus the PLIC plane can exceed 16 loops (FMFPA on hexahedra: 13 + 6 + 1);
and the autotuner's choice of faces per warp and of prebuilt polyhedra keeps
the results."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vof():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, vof as V
    build.build()
    return V


def _case(name):
    if name == "hex":
        m = I.hex_mesh(16)
        return m, I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15), levels=3), \
            I.deformation(3.0), 0.5
    if name == "hex7":  # coarse cells, a large interface: many cells cut per polyhedron
        m = I.hex_mesh(7)
        return m, I.init_fraction(m, I.sphere((0.45, 0.5, 0.52), 0.3), levels=3), \
            I.deformation(3.0), 0.5
    m = I.kuhn_tet_mesh(5, seed=3)
    return m, I.init_fraction(m, I.sphere((0.5, 0.6, 0.5), 0.25), levels=3), \
        I.rotation(2 * np.pi), 0.4


@pytest.mark.parametrize("name,flux", [("hex", "NMFPA"), ("hex7", "NMFPA"), ("tet", "FMFPA"),
                                       ("tet", "NMFPA")])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_half_warp_faces_are_bit_identical(vof, name, flux, prec):
    m, F0, vel, cfl = _case(name)
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    kw = dict(precision=P, flux=getattr(vof, "FLUX_" + flux))
    one = vof.Context(m, faces_per_warp=1, **kw)
    two = vof.Context(m, faces_per_warp=2, **kw)
    for c in (one, two):
        c.set_fraction(F0)
        c.reconstruct()
    t = 0.0
    for _ in range(6):
        dt = one.suggest_dt(vel, t, cfl, 10.0)
        one.step(vel, t, dt)
        two.step(vel, t, dt)
        t += dt
        assert np.array_equal(one.face_flux()[1], two.face_flux()[1])
        assert np.array_equal(one.get_fraction(), two.get_fraction())
    s1, s2 = one.stats(), two.stats()
    assert s1["n_active_faces"] > 100 and s2["n_overflow"] == 0
    assert s1["n_truncations"] == s2["n_truncations"]


def test_half_warp_is_refused_where_it_does_not_fit(vof):
    m = I.trihex_mesh(3, seed=2)  # non-convex cells of 24 faces
    with pytest.raises(vof.VofError) as e:
        vof.Context(m, faces_per_warp=2)
    assert e.value.status == vof.VOF_EINVAL
    with pytest.raises(vof.VofError):
        vof.Context(I.hex_mesh(4), flux=vof.FLUX_EMFPA, faces_per_warp=2)
    with pytest.raises(vof.VofError):
        vof.Context(I.hex_mesh(4), faces_per_warp=2)  # FMFPA: 13 + 6 + 1 loops
    vof.Context(I.hex_mesh(4), flux=vof.FLUX_NMFPA, faces_per_warp=2)
    vof.Context(I.kuhn_tet_mesh(2, seed=1), faces_per_warp=2)
    with pytest.raises(vof.VofError):
        vof.Context(I.hex_mesh(4), faces_per_warp=3)
    vof.Context(m)  # the library's choice falls back to whole warps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_knobs_keep_results(vof, prec):
    m, F0, vel, cfl = _case("tet")
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    a = vof.Context(m, precision=P)
    b = vof.Context(m, precision=P, faces_per_warp=1)
    for c in (a, b):
        c.set_fraction(F0)
        c.reconstruct()
    dt = a.suggest_dt(vel, 0.0, cfl, 10.0)
    fb, rb, fw, pb = a.autotune(vel, 0.0, dt, full=True)
    assert fw in (1, 2) and pb in (0, 1) and fb % 152 == 0 and rb % 152 == 0
    t = 0.0
    for _ in range(3):
        dt = a.suggest_dt(vel, t, cfl, 10.0)
        a.step(vel, t, dt)
        b.step(vel, t, dt)
        t += dt
    assert np.array_equal(a.get_fraction(), b.get_fraction())

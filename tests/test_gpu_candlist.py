"""Candidate lists built ahead of the flux kernel (FP32 path, hexahedral
grids): the flux kernel reads each prebuilt polyhedron's list of candidate
cells instead of searching the two node-neighbour rings itself. The list
kernel runs the same filter in the same order, so the results are the same
bit for bit whether a face's list comes prebuilt or the flux kernel searches
(faces past the prebuilt capacity), and tetrahedral grids (many node
neighbours) build no lists at all."""
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


@pytest.mark.parametrize("flux", ["FMFPA", "EMFPA", "NMFPA"])
@pytest.mark.parametrize("grid", ["hex", "trihex"])
def test_prebuilt_lists_equal_the_kernel_search(vof, flux, grid):
    if grid == "hex":
        m = I.hex_mesh(16)
        F0 = I.init_fraction(m, I.sphere((0.45, 0.5, 0.5), 0.28), levels=3)
        vel, cfl = I.deformation(3.0), 0.5
    else:
        m = I.trihex_mesh(6, seed=3)
        F0 = I.init_fraction(m, I.sphere((0.5, 0.48, 0.52), 0.3), levels=3)
        vel, cfl = I.translation((0.2, -0.1, 0.05)), 0.5
    kw = dict(precision=vof.PREC_MIXED, flux=getattr(vof, "FLUX_" + flux))
    full = vof.Context(m, **kw)                  # every active face prebuilt with its list
    few = vof.Context(m, poly_capacity=7, **kw)  # 7 faces prebuilt, the rest searched in the kernel
    for c in (full, few):
        c.set_fraction(F0)
        c.reconstruct()
    t = 0.0
    for _ in range(6):
        dt = full.suggest_dt(vel, t, cfl, 10.0)
        full.step(vel, t, dt)
        few.step(vel, t, dt)
        t += dt
        assert np.array_equal(full.face_flux()[1], few.face_flux()[1])
        assert np.array_equal(full.get_fraction(), few.get_fraction())
    s1, s2 = full.stats(), few.stats()
    assert s1["n_active_faces"] > 100 and s1["n_truncations"] == s2["n_truncations"]
    assert s1["n_overflow"] == 0


def test_lists_are_built_on_hex_grids_only(vof):
    """The list kernel is one more launch of the polyhedra phase on a hex
    grid (mixed precision) and none on tetrahedra or in FP64."""
    def polyhedra_launches(m, prec):
        c = vof.Context(m, precision=prec)
        c.set_fraction(np.full(int(m["n_cell"]), 0.5))
        c.reconstruct()
        c.set_timing(True)
        c.advect(I.translation((0.3, 0.2, 0.1)), 0.0, 1e-3)
        return c.timing()["polyhedra"][1]
    hexm = I.hex_mesh(6)
    tetm = I.kuhn_tet_mesh(3, seed=2)
    assert polyhedra_launches(hexm, vof.PREC_MIXED) == 2
    assert polyhedra_launches(tetm, vof.PREC_MIXED) == 1
    assert polyhedra_launches(hexm, vof.PREC_FP64) == 1

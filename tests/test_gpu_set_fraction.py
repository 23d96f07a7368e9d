"""vof_set_fraction between steps, through the C-ABI.

Setting F keeps the band-limited sweeps when only cells of the last advect's
band change, and makes them full otherwise; either way the next steps must be
those of full sweeps. References: a context that never leaves the device
(round trip), and a fresh context given the same F (every sweep full).
F, tags and planes are compared bit for bit.
"""
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


@pytest.fixture(scope="module")
def case():
    m = I.hex_mesh(24)
    return m, I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15), levels=3)


VEL = I.deformation(3.0)
DT = 0.02


def _same(a, b, face_tags=True):
    """F, node / face / cell tags and planes bit for bit (face tags come from
    the face sweep of an advect, so a context that has only reconstructed
    has none to compare)"""
    Fa, Fb = a.get_fraction(), b.get_fraction()
    assert np.array_equal(Fa, Fb)
    (va, fa, ca), (vb, fb, cb) = a.tags(), b.tags()
    assert np.array_equal(va, vb) and np.array_equal(ca, cb)
    if face_tags:
        assert np.array_equal(fa, fb)
    assert np.array_equal(a.planes(), b.planes())


def _ctx(vof, m, F, prec):
    c = vof.Context(m, precision=prec)
    c.set_fraction(F)
    c.reconstruct()
    return c


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mem", ["host", "device"])
def test_round_trip_each_step_changes_nothing(vof, case, prec, mem):
    """Reading F back and setting it again before every step (what a caller
    holding F on the host does) leaves every result bit-identical to the
    run that stays on the device."""
    import torch
    m, F0 = case
    p = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    a, b = _ctx(vof, m, F0, p), _ctx(vof, m, F0, p)
    t = 0.0
    for _ in range(6):
        a.advect(VEL, t, DT)
        b.advect(VEL, t, DT)
        F = b.get_fraction()
        b.set_fraction(F if mem == "host" else torch.from_numpy(F).cuda())
        a.reconstruct()
        b.reconstruct()
        t += DT
    _same(a, b)
    s = b.stats()
    assert s["n_overflow"] == 0


@pytest.mark.parametrize("where", ["outside", "band", "both"])
def test_changed_cells_give_full_sweep_results(vof, case, where):
    """After some steps, F is changed in a uniform cell far from the body
    (outside the band: the next sweeps must be full), in interfacial cells
    (inside the band: they may stay band-limited), or both. The continued
    context then steps exactly like a fresh one given the same F."""
    m, F0 = case
    p = vof.PREC_MIXED
    a = _ctx(vof, m, F0, p)
    t = 0.0
    for _ in range(4):
        a.step(VEL, t, DT)
        t += DT
    a.advect(VEL, t, DT)
    t += DT
    F = a.get_fraction()
    n = 24
    if where in ("outside", "both"):
        far = (n - 2) * n * n + (n - 2) * n + (n - 2)  # near the corner (1, 1, 1)
        assert F[far] == 0.0
        F[far] = 0.3
    if where in ("band", "both"):
        inter = np.flatnonzero((F > 0.05) & (F < 0.95))[:5]
        assert inter.size == 5
        F[inter] *= 0.97
    a.set_fraction(F)
    a.reconstruct()
    b = _ctx(vof, m, F, p)
    _same(a, b, face_tags=False)
    for _ in range(3):
        a.step(VEL, t, DT)
        b.step(VEL, t, DT)
        t += DT
    _same(a, b)


def test_set_fraction_restarts_bookkeeping(vof, case):
    """The volume bookkeeping of vof_stats counts from the last set F."""
    m, F0 = case
    a = _ctx(vof, m, F0, vof.PREC_FP64)
    t = 0.0
    for _ in range(3):
        a.step(VEL, t, DT)
        t += DT
    F = a.get_fraction()
    a.set_fraction(F)
    s = a.stats()
    assert s["clip_loss"] == 0.0 and s["cutoff_loss"] == 0.0 and s["boundary_outflow"] == 0.0

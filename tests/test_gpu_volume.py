"""Volume bookkeeping of both paths (Sec. 2.2, Eq. fnext and the final clip;
Sec. 2.1 cut-off).

The update moves fluid between cells by face volumes applied with opposite
signs to the two cells of a face, so the total changes only by what the clip
to [0, 1] and the cut-off remove and by what leaves through the domain
boundary. The library sums those three terms (each in a fixed order); the
identity V(t) = V0 - clip - cutoff - boundary must hold to rounding in the
FP64 path and in the mixed path alike (the mixed path's FP32 flux noise shows
up as clip loss, not as unaccounted volume).
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


def _cases():
    m = I.hex_mesh(12)
    yield "hex12-deformation", m, I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15), levels=4), \
        I.deformation(3.0), 0.5
    # a body that leaves the domain through x = 1: boundary outflow
    yield "hex12-outflow", m, I.init_fraction(m, I.sphere((0.8, 0.5, 0.5), 0.15), levels=4), \
        I.translation((1.0, 0.2, 0.0)), 0.5
    m = I.kuhn_tet_mesh(4, seed=4)
    yield "tet4-rotation", m, I.init_fraction(m, I.sphere((0.5, 0.6, 0.5), 0.3), levels=3), \
        I.rotation(2 * np.pi), 0.4
    m = I.trihex_mesh(3, seed=6)
    yield "trihex3-translation", m, I.init_fraction(m, I.ellipsoid((0.6, 0.5, 0.5), (0.3, 0.2, 0.25)),
                                                   levels=3), I.translation((0.6, -0.3, 0.2)), 0.5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_volume_bookkeeping(vof, prec):
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    for name, m, F0, vel, cfl in _cases():
        ctx = vof.Context(m, precision=P)
        ctx.set_fraction(F0)
        V = ctx.geometry()["cell_vol"]
        vol0 = float((V * F0).sum())
        ctx.reconstruct()
        t = 0.0
        for _ in range(25):
            dt = ctx.suggest_dt(vel, t, cfl, 10.0)
            ctx.step(vel, t, dt)
            t += dt
        s = ctx.stats()
        resid = s["volume"] - (vol0 - s["clip_loss"] - s["cutoff_loss"] - s["boundary_outflow"])
        assert abs(resid) < 1e-12 * vol0, (name, resid / vol0, s)
        if name == "hex12-outflow":
            assert s["boundary_outflow"] > 1e-3 * vol0, s
        # the F that the context reports agrees with its own volume sum
        assert abs(float((V * ctx.get_fraction()).sum()) - s["volume"]) < 1e-13 * vol0

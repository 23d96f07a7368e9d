"""Candidate-ring escape detection (Sec. 2.2 with the CFL condition of
Sec. 3.3): the flux of a face is truncated against the cells around it (its
owner, its neighbour and their node neighbours), which cover the flux
polyhedron only while the time step is small enough. On the jittered Kuhn
tetrahedra in rigid rotation, the oracle's polyhedra of 13 active faces have
a vertex inside the domain but in none of those cells at CFL 0.8 and none at
CFL 0.6 or below (found by exact point-in-cell tests on the CPU). The library
counts such polyhedra on the device and reports VOF_ECFL from
vof_get_stats."""
import ctypes

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
    m = I.kuhn_tet_mesh(6, seed=4)
    F0 = I.init_fraction(m, I.sphere((0.5, 0.5, 0.5), 0.33), levels=3)
    return m, F0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("flux", ["FMFPA", "EMFPA", "NMFPA"])
def test_escape_is_counted_and_reported(vof, case, prec, flux):
    m, F0 = case
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    vel = I.rotation(2 * np.pi)
    ctx = vof.Context(m, precision=P, flux=getattr(vof, "FLUX_" + flux))
    ctx.set_fraction(F0)
    ctx.reconstruct()
    st = ctx.get_state()
    counts = {}
    for cfl in (0.4, 0.5, 0.8):
        ctx.set_state(st)
        dt = ctx.suggest_dt(vel, 0.0, cfl, 1e9)
        ctx.advect(vel, 0.0, dt)
        s = vof.Stats()
        status = vof.lib().vof_get_stats(ctx._h, ctypes.byref(s), None)
        counts[cfl] = s.n_escaped
        assert s.n_active_faces > 1000
        if s.n_escaped:
            assert status == vof.VOF_ECFL
            assert b"candidate" in vof.lib().vof_last_error()
            assert ctx.stats()["cfl_escape"]
            with pytest.raises(vof.VofError) as e:
                ctx.stats(raise_on_escape=True)
            assert e.value.status == vof.VOF_ECFL
        else:
            assert status == vof.VOF_OK
    assert counts[0.4] == 0 and counts[0.5] == 0, counts
    if flux == "FMFPA":
        assert counts[0.8] >= 5, counts
    else:
        assert counts[0.8] >= 1, counts


def test_paper_workloads_do_not_escape(vof):
    """The hex deformation at CFL 0.5 and the jittered tets in rotation at
    CFL 0.4 (the paper's workloads here) stay inside the candidate ring for
    10 steps."""
    for m, body, vel, cfl in [
            (I.hex_mesh(24), I.sphere((0.35, 0.35, 0.35), 0.15), I.deformation(3.0), 0.5),
            (I.kuhn_tet_mesh(6, seed=4), I.sphere((0.5, 0.75, 0.5), 0.15), I.rotation(2 * np.pi),
             0.4)]:
        for P in (vof.PREC_FP64, vof.PREC_MIXED):
            ctx = vof.Context(m, precision=P)
            ctx.set_fraction(I.init_fraction(m, body, levels=3))
            ctx.reconstruct()
            t = 0.0
            for _ in range(10):
                dt = ctx.suggest_dt(vel, t, cfl, 10.0)
                ctx.step(vel, t, dt)
                t += dt
                assert ctx.stats()["n_escaped"] == 0

"""Batching, CUDA-graph replay and the launch-shape autotuner.

A grid advanced inside a batch runs the same per-face and per-cell
arithmetic as alone, so its results must be bit-identical to the single-grid
run; so must a graph replay of a step and a step after autotuning.
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


def _grids():
    g = []
    m = I.hex_mesh(10)
    g.append((m, I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.2), levels=3), I.deformation(3.0)))
    m = I.kuhn_tet_mesh(3, seed=4)
    g.append((m, I.init_fraction(m, I.sphere((0.5, 0.6, 0.5), 0.3), levels=3), I.rotation(2 * np.pi)))
    m = I.trihex_mesh(3, seed=6)
    g.append((m, I.init_fraction(m, I.ellipsoid((0.5, 0.5, 0.5), (0.3, 0.2, 0.25)), levels=3),
              I.translation((0.6, -0.3, 0.2))))
    return g


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_is_bit_identical_to_single_grids(vof, prec):
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    grids = _grids()
    batch = vof.Context([m for m, _, _ in grids], precision=P)
    batch.set_fraction(np.concatenate([F for _, F, _ in grids]))
    batch.reconstruct()
    singles = []
    for m, F, _ in grids:
        c = vof.Context(m, precision=P)
        c.set_fraction(F)
        c.reconstruct()
        singles.append(c)
    vels = [v for _, _, v in grids]
    t = np.zeros(len(grids))
    for _ in range(3):
        dt = batch.suggest_dt_batch(vels, t, 0.5, np.full(len(grids), 10.0))
        for i, c in enumerate(singles):
            assert c.suggest_dt(vels[i], t[i], 0.5, 10.0) == dt[i]
            c.step(vels[i], t[i], dt[i])
        batch.step_batch(vels, t, dt)
        t = t + dt
    Fb = batch.get_fraction()
    Vd, VF = batch.face_flux()
    for i, c in enumerate(singles):
        a, b = batch.cell_off[i], batch.cell_off[i + 1]
        assert np.array_equal(Fb[a:b], c.get_fraction()), i
        fa, fb = batch.face_off[i], batch.face_off[i + 1]
        vd1, vf1 = c.face_flux()
        assert np.array_equal(VF[fa:fb], vf1) and np.array_equal(Vd[fa:fb], vd1), i
    assert batch.stats()["n_overflow"] == 0


def test_graph_replay_matches_launches(vof):
    import torch
    grids = _grids()[:2]
    meshes = [m for m, _, _ in grids]
    F0 = np.concatenate([F for _, F, _ in grids])
    vels = [v for _, _, v in grids]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = vof.Context(meshes, precision=vof.PREC_MIXED)
        b = vof.Context(meshes, precision=vof.PREC_MIXED)
        for c in (a, b):
            c.set_fraction(F0)
            c.reconstruct()
        t = np.zeros(2)
        dt0 = a.suggest_dt_batch(vels, t, 0.5, np.full(2, 10.0))
        a.graph_capture(with_reconstruct=True)
        for _ in range(4):
            dt = a.suggest_dt_batch(vels, t, 0.5, np.full(2, 10.0))
            a.graph_launch(vels, t, dt)
            b.step_batch(vels, t, dt)
            t = t + dt
        Fa, Fb = a.get_fraction(), b.get_fraction()
    assert dt0[0] > 0
    assert np.array_equal(Fa, Fb)
    assert not np.array_equal(Fa, F0)


def test_autotune_keeps_results(vof):
    grids = _grids()
    meshes = [m for m, _, _ in grids]
    F0 = np.concatenate([F for _, F, _ in grids])
    vels = [v for _, _, v in grids]
    a = vof.Context(meshes, precision=vof.PREC_MIXED)
    b = vof.Context(meshes, precision=vof.PREC_MIXED)
    for c in (a, b):
        c.set_fraction(F0)
        c.reconstruct()
    t = np.zeros(3)
    dt = a.suggest_dt_batch(vels, t, 0.5, np.full(3, 10.0))
    fb, rb = a.autotune(vels, t, dt)
    assert fb % 152 == 0 and rb % 152 == 0 and 2 * 152 <= fb <= 16 * 152
    assert np.array_equal(a.get_fraction(), b.get_fraction())
    for _ in range(2):
        dt = a.suggest_dt_batch(vels, t, 0.5, np.full(3, 10.0))
        a.step_batch(vels, t, dt)
        b.step_batch(vels, t, dt)
        t = t + dt
    assert np.array_equal(a.get_fraction(), b.get_fraction())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_a_grid_that_pauses_keeps_its_state_and_resumes_exactly(vof, prec):
    """A grid of a batch that takes dt = 0 for some steps (a served request
    that is done, or waits) keeps F bit for bit, costs no flux polyhedra,
    and when it moves again continues exactly as a single grid that simply
    skipped those steps; the other grids are unaffected."""
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    grids = _grids()
    vels = [v for _, _, v in grids]
    batch = vof.Context([m for m, _, _ in grids], precision=P)
    batch.set_fraction(np.concatenate([F for _, F, _ in grids]))
    batch.reconstruct()
    singles = []
    for m, F, _ in grids:
        c = vof.Context(m, precision=P)
        c.set_fraction(F)
        c.reconstruct()
        singles.append(c)
    n = len(grids)
    t = np.zeros(n)
    pause = 1  # the tet grid stops for steps 2..4
    for k in range(7):
        dt = batch.suggest_dt_batch(vels, t, 0.5, np.full(n, 10.0))
        if 2 <= k <= 4:
            dt[pause] = 0.0
        for i, c in enumerate(singles):
            if dt[i] > 0.0:
                c.step(vels[i], t[i], dt[i])
        before = batch.get_fraction()
        batch.step_batch(vels, t, dt)
        after = batch.get_fraction()
        t = t + dt
        Fb = np.split(after, np.cumsum([int(m["n_cell"]) for m, _, _ in grids])[:-1])
        for i, c in enumerate(singles):
            assert np.array_equal(Fb[i], c.get_fraction()), (k, i)
        if 2 <= k <= 4:
            Fp = np.split(before, np.cumsum([int(m["n_cell"]) for m, _, _ in grids])[:-1])[pause]
            assert np.array_equal(Fb[pause], Fp)
    assert batch.stats()["n_overflow"] == 0

"""Serving on the GPU: requests that arrive while others run are admitted and
overlap on the device; each result is the same alone and in the mix."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01524_gb300 import build, serve, vof
    build.build()
    return vof, serve


def _requests(serve):
    specs = [
        (I.hex_mesh(12), I.sphere((0.35, 0.35, 0.35), 0.2), I.deformation(3.0), 8, 0.000),
        (I.kuhn_tet_mesh(3, seed=2), I.sphere((0.5, 0.6, 0.5), 0.3), I.rotation(2 * np.pi), 6, 0.002),
        (I.trihex_mesh(3, seed=4), I.ellipsoid((0.5, 0.5, 0.5), (0.3, 0.2, 0.25)),
         I.translation((0.5, -0.4, 0.3)), 7, 0.004),
        (I.hex_mesh(10), I.sphere((0.5, 0.5, 0.5), 0.25), I.translation((-0.3, 0.2, 0.6)), 9, 0.004),
    ]
    out = []
    for rid, (m, body, vel, n, arr) in enumerate(specs):
        F0 = I.init_fraction(m, body, levels=3)
        out.append(serve.Request(rid=rid, mesh=m, F0=F0, vel=vel, n_steps=n, arrival=arr))
    return out


def _alone(vof, r, prec):
    c = vof.Context(r.mesh, precision=prec)
    c.set_fraction(r.F0)
    c.reconstruct()
    t = 0.0
    for _ in range(r.n_steps):
        dt = c.suggest_dt(r.vel, t, r.cfl, r.t_end)
        c.step(r.vel, t, dt)
        t += dt
    return c.get_fraction()


@pytest.mark.parametrize("graphs", [True, False])
def test_results_alone_and_in_the_mix(env, graphs):
    vof, serve = env
    reqs = _requests(serve)
    backend = serve.DeviceBackend(precision_mixed=True, use_graphs=graphs)
    st = serve.Server(backend).run(reqs)
    s = st.summary()
    assert s["requests"] == 4 and s["max_active"] >= 2
    for r in reqs:
        assert r.result is not None and r.t_done >= r.t_admit >= r.arrival
        assert np.array_equal(r.result, _alone(vof, r, vof.PREC_MIXED)), r.rid


def test_budget_limits_residency(env):
    vof, serve = env
    reqs = _requests(serve)
    # a budget that holds the largest request alone: requests wait for room,
    # the resident set never exceeds the budget, and every result is right
    big = max(serve.estimate_device_bytes(r.mesh) for r in reqs)
    st = serve.Server(serve.DeviceBackend(), budget_bytes=big).run(reqs)
    assert st.max_bytes <= big and st.summary()["max_active"] < len(reqs)
    for r in reqs:
        assert np.array_equal(r.result, _alone(vof, r, vof.PREC_MIXED))

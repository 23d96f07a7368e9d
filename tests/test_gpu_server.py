"""The device-resident serving loop (vof_server_*) on the GPU: requests that
arrive while others run are admitted as slots of new batched contexts, their
work overlaps on the device, the device-byte budget binds, and each result
equals the request run alone, bit for bit. Also: vof_estimate_bytes, which
the server admits against, equals what a context allocates."""
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


def _specs():
    return [
        (I.hex_mesh(12), I.sphere((0.35, 0.35, 0.35), 0.2), I.deformation(3.0), 8, 0.5),
        (I.kuhn_tet_mesh(3, seed=2), I.sphere((0.5, 0.6, 0.5), 0.3), I.rotation(2 * np.pi), 6, 0.4),
        (I.trihex_mesh(3, seed=4), I.ellipsoid((0.5, 0.5, 0.5), (0.3, 0.2, 0.25)),
         I.translation((0.5, -0.4, 0.3)), 7, 0.5),
        (I.hex_mesh(10), I.sphere((0.5, 0.5, 0.5), 0.25), I.translation((-0.3, 0.2, 0.6)), 9, 0.5),
        (I.kuhn_tet_mesh(4, seed=5), I.sphere((0.45, 0.5, 0.55), 0.25), I.deformation(3.0), 5, 0.4),
    ]


def _alone(vof, m, F0, vel, n, cfl):
    c = vof.Context(m, precision=vof.PREC_MIXED)
    c.set_fraction(F0)
    c.reconstruct()
    t = 0.0
    for _ in range(n):
        dt = c.suggest_dt(vel, t, cfl, 1e9)
        c.step(vel, t, dt)
        t += dt
    return c.get_fraction()


def test_results_alone_and_in_the_mix(vof):
    """Three requests submitted at once, two more while those run: five
    slots in two contexts, and every result equal to the request run alone."""
    specs = _specs()
    F0s = [I.init_fraction(m, b, levels=3) for m, b, _, _, _ in specs]
    srv = vof.Server(budget_bytes=0, precision=vof.PREC_MIXED)
    ids = [srv.submit(m, F0, vel, n, cfl) for (m, _, vel, n, cfl), F0 in zip(specs[:3], F0s)]
    for _ in range(2):
        srv.step()
    ids += [srv.submit(m, F0, vel, n, cfl) for (m, _, vel, n, cfl), F0 in zip(specs[3:], F0s[3:])]
    srv.drain()
    st = srv.stats()
    assert st["n_done"] == 5 and st["n_batches"] == 2 and st["max_active"] == 5
    assert st["device_bytes"] == 0 and st["peak_device_bytes"] > 0
    assert st["cell_steps"] == sum(int(m["n_cell"]) * n for m, _, _, n, _ in specs)
    for rid, (m, _, vel, n, cfl), F0 in zip(ids, specs, F0s):
        state, F, lat = srv.poll(rid)
        assert state == vof.REQ_DONE and lat > 0
        assert np.array_equal(F, _alone(vof, m, F0, vel, n, cfl)), rid


def test_budget_binds_and_results_stay_exact(vof):
    """A budget that holds the largest request alone: requests wait for room,
    the live contexts never exceed it, and every result is exact."""
    specs = _specs()
    F0s = [I.init_fraction(m, b, levels=3) for m, b, _, _, _ in specs]
    big = max(vof.estimate_bytes(m, vof.PREC_MIXED) for m, _, _, _, _ in specs)
    srv = vof.Server(budget_bytes=big, precision=vof.PREC_MIXED)
    ids = [srv.submit(m, F0, vel, n, cfl) for (m, _, vel, n, cfl), F0 in zip(specs, F0s)]
    srv.drain()
    st = srv.stats()
    assert st["peak_device_bytes"] <= big and st["n_batches"] >= 2
    assert st["max_active"] < len(specs)
    for rid, (m, _, vel, n, cfl), F0 in zip(ids, specs, F0s):
        assert np.array_equal(srv.poll(rid)[1], _alone(vof, m, F0, vel, n, cfl)), rid
    # a request above the budget alone is refused with a message
    small = vof.Server(budget_bytes=1024, precision=vof.PREC_MIXED)
    small.submit(specs[0][0], F0s[0], specs[0][2], 2, 0.5)
    with pytest.raises(vof.VofError) as e:
        small.step()
    assert e.value.status == vof.VOF_ENOMEM and "budget" in str(e.value)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_estimate_bytes_equals_the_allocation(vof, prec):
    P = vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED
    meshes = [I.hex_mesh(7), I.kuhn_tet_mesh(3, seed=1), I.trihex_mesh(2, seed=3)]
    for kw in ({}, {"recon": vof.RECON_LSFIR}, {"flux": vof.FLUX_EMFPA}, {"poly_capacity": 17}):
        for ms in ([meshes[0]], [meshes[1]], [meshes[2]], meshes):
            c = vof.Context(ms if len(ms) > 1 else ms[0], precision=P, **kw)
            assert vof.estimate_bytes(ms, P, **kw) == c.device_bytes, (prec, kw, len(ms))
            c.close()

"""Checkpoint / resume and determinism through the C-ABI: k steps, save,
restore into a new context of the same mesh, the remaining steps -- F and the
planes bit for bit the uninterrupted run, for both precisions and the
non-default constructions (the volume bookkeeping to rounding: its per-block
partial sums follow the sweep's assignment of cells to blocks, and the first
sweeps after a restore are full); two identical runs give identical bits;
bad states are refused."""
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


def _run(ctx, vel, t0, n, dt=0.02):
    t = t0
    for _ in range(n):
        ctx.step(vel, t, dt)
        t += dt
    return t


@pytest.mark.parametrize("setting", ["fp64", "mixed", "mixed-emfpa-lsfir", "fp64-nmfpa-tets"])
def test_resume_is_bit_identical(vof, setting):
    if setting == "fp64-nmfpa-tets":
        m = I.kuhn_tet_mesh(4, seed=3)
        F0 = I.init_fraction(m, I.sphere((0.5, 0.55, 0.5), 0.27), levels=3)
    else:
        m = I.hex_mesh(12)
        F0 = I.init_fraction(m, I.sphere((0.35, 0.35, 0.35), 0.15), levels=3)
    kw = {"precision": vof.PREC_MIXED if setting.startswith("mixed") else vof.PREC_FP64}
    if "emfpa" in setting:
        kw["flux"] = vof.FLUX_EMFPA
    if "nmfpa" in setting:
        kw["flux"] = vof.FLUX_NMFPA
    if "lsfir" in setting:
        kw["recon"] = vof.RECON_LSFIR
    vel = I.deformation(3.0)
    a = vof.Context(m, **kw)
    a.set_fraction(F0)
    a.reconstruct()
    t = _run(a, vel, 0.0, 3)
    state = a.get_state()
    _run(a, vel, t, 4)
    b = vof.Context(m, **kw)
    b.set_state(state)
    _run(b, vel, t, 4)
    assert np.array_equal(a.get_fraction(), b.get_fraction())
    assert np.array_equal(a.planes(), b.planes())
    sa, sb = a.stats(), b.stats()
    assert sa["volume"] == sb["volume"] and sa["n_interfacial"] == sb["n_interfacial"]
    for k in ("clip_loss", "cutoff_loss", "boundary_outflow"):
        assert abs(sa[k] - sb[k]) <= 1e-14 * sa["volume"], k


def test_two_runs_are_bit_identical(vof):
    """Determinism (the check that stands in for a race detector here):
    every sum is formed in a fixed order, so two runs agree to the bit."""
    m = I.trihex_mesh(3, seed=2)
    F0 = I.init_fraction(m, I.sphere((0.5, 0.48, 0.52), 0.3), levels=3)
    out = []
    for _ in range(2):
        c = vof.Context(m, precision=vof.PREC_MIXED)
        c.set_fraction(F0)
        c.reconstruct()
        _run(c, I.rotation(2 * np.pi), 0.0, 5)
        out.append((c.get_fraction(), c.planes(), c.stats()["volume"]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_bad_states_are_refused(vof):
    m = I.hex_mesh(6)
    c = vof.Context(m)
    c.set_fraction(np.full(m["n_cell"], 0.5))
    with pytest.raises(vof.VofError) as e:
        c.get_state()  # no reconstruction yet
    assert e.value.status == vof.VOF_ESTATE
    c.reconstruct()
    st = c.get_state()
    other = vof.Context(I.hex_mesh(7))
    with pytest.raises(vof.VofError) as e:
        other.set_state(st)
    assert e.value.status == vof.VOF_EINVAL
    bad = st.copy()
    bad[0] ^= 0xFF
    with pytest.raises(vof.VofError):
        c.set_state(bad)
    with pytest.raises(vof.VofError):
        c.set_state(st[:100])
    short = np.empty(10, np.uint8)
    assert vof.lib().vof_get_state(c._h, vof._ptr(short), short.size, None, None) == vof.VOF_EINVAL

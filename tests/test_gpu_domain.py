"""Partitioned grid on one GPU: the parts are library contexts on their
sub-meshes (owned cells plus a halo of node rings), and the halo exchange is
a device-to-device copy between them (gather over the sending part's list,
scatter into the receiving part's halo). With the halo depth
``partition.halo_rings`` gives for the options, every owned cell's F equals
the unpartitioned context's bit for bit over coupled steps, for the FP64 and
mixed paths, LSGIR and LSFIR, the three flux polyhedra, hex and tetrahedral
grids, two slabs and three bisected parts; the time step from bounds reduced
over the parts equals the whole grid's, and the sum of the parts' owned
volumes matches the whole grid's."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import domain as D
from paper_2111_01524_gb300 import inputs as I
from paper_2111_01524_gb300 import partition as P

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
        m = I.hex_mesh(20)
        F0 = I.init_fraction(m, I.sphere((0.5, 0.45, 0.52), 0.3), levels=3)
        return m, F0, I.deformation(3.0), 0.5
    m = I.kuhn_tet_mesh(8, seed=3)
    F0 = I.init_fraction(m, I.sphere((0.5, 0.55, 0.5), 0.27), levels=3)
    return m, F0, I.rotation(2 * np.pi), 0.4


CASES = [
    ("hex", 2, "fp64", "FMFPA", 0),
    ("hex", 2, "mixed", "FMFPA", 0),
    ("hex", 3, "fp64", "EMFPA", 0),
    ("hex", 3, "mixed", "NMFPA", 1),
    ("hex", 2, "fp64", "FMFPA", 1),
    ("tet", 2, "mixed", "FMFPA", 0),
    ("tet", 3, "fp64", "NMFPA", 0),
]


@pytest.mark.parametrize("name,n_parts,prec,flux,recon", CASES)
def test_partitioned_grid_is_bit_identical(vof, name, n_parts, prec, flux, recon):
    m, F0, vel, cfl = _case(name)
    kw = dict(precision=vof.PREC_FP64 if prec == "fp64" else vof.PREC_MIXED,
              flux=getattr(vof, "FLUX_" + flux), recon=recon)
    whole = vof.Context(m, **kw)
    whole.set_fraction(F0)
    whole.reconstruct()
    part = P.slab_partition(m, n_parts) if n_parts == 2 else P.rcb_partition(m, n_parts)
    pg = D.PartitionedGrid(m, part=part, **kw)
    assert pg.rings == P.halo_rings(kw["precision"], recon, 4)
    pg.set_fraction(F0)
    pg.reconstruct()
    t = 0.0
    for k in range(10):
        dt = whole.suggest_dt(vel, t, cfl, 10.0)
        assert pg.suggest_dt(vel, t, cfl, 10.0) == dt
        whole.step(vel, t, dt)
        pg.step(vel, t, dt)
        t += dt
        Fw = whole.get_fraction()
        Fp = pg.get_fraction()
        assert np.array_equal(Fp, Fw), (k, np.abs(Fp - Fw).max())
    st = whole.stats()
    assert abs(pg.volume() - st["volume"]) <= 1e-13 * st["volume"]
    # the interface crossed into the halos
    n_int = 0
    for sd, pt in zip(pg.subs, pg.parts):
        F = pt.fraction()
        h = sd.ring > 0
        n_int += int(np.sum((F[h] > 0) & (F[h] < 1)))
    assert n_int > 0


def test_halo_calls_check_their_arguments(vof):
    import torch
    m = I.hex_mesh(4)
    c = vof.Context(m)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(vof.VofError) as e:  # no lists yet
        vof._check(vof.lib().vof_halo_import(c._h, 0, buf.data_ptr(), None))
    assert e.value.status == vof.VOF_ESTATE
    with pytest.raises(vof.VofError):
        c.set_lists([np.array([0, 64], np.int32)])  # 64 is not a cell
    c.set_lists([np.arange(8, dtype=np.int32), np.zeros(0, np.int32)])
    c.set_fraction(np.full(64, 0.25))
    c.export_list(0, buf)
    assert torch.all(buf == 0.25)
    c.import_list(0, torch.full((8,), 0.5, dtype=torch.float64, device="cuda"))
    F = c.get_fraction()
    assert np.all(F[:8] == 0.5) and np.all(F[8:] == 0.25)
    assert c.list_volume(0) == pytest.approx(8 * 0.5 / 64, rel=1e-15)
    assert c.list_volume(1) == 0.0
    with pytest.raises(vof.VofError):
        c.list_volume(2)
    with pytest.raises(vof.VofError) as e:
        c.step(I.rotation(1.0), 0.0, 1e-3)  # the import needs a reconstruction first
    assert e.value.status == vof.VOF_ESTATE

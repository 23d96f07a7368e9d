"""Domain decomposition of one grid, on CPU: partition and halo properties,
and the partitioned step against the whole grid's, with the oracle as each
part's stepper (the host logic is the library's: the partition, the halo
lists, the exchange order and the reductions).

A part is a sub-mesh of its owned cells plus ``rings`` node rings; every
step the parts advect, the halo cells receive F from their owners, and the
parts reconstruct. With the halo depth ``partition.halo_rings`` gives, the
owned cells' F equals the whole grid's bit for bit, in one process (two and
three parts) and over two gloo ranks (point-to-point halo exchange,
all-reduced time-step bounds and volume). One ring is too shallow: the
partitioned F then departs from the whole grid's, which shows the comparison
can fail.
"""
import os
import socket

import numpy as np
import pytest

from paper_2111_01524_gb300 import domain as D
from paper_2111_01524_gb300 import inputs as I
from paper_2111_01524_gb300 import partition as P


# ---------------------------------------------------------------- partition
def _grids():
    hex_m = I.hex_mesh(10)
    tet_m = I.kuhn_tet_mesh(4, seed=3)
    tri_m = I.trihex_mesh(3, seed=2)
    return {"hex": hex_m, "tet": tet_m, "trihex": tri_m}


@pytest.mark.parametrize("name", ["hex", "tet", "trihex"])
@pytest.mark.parametrize("n_parts,method", [(2, "slab"), (3, "rcb"), (4, "rcb")])
def test_parts_cover_the_grid_and_halos_are_rings(name, n_parts, method):
    m = _grids()[name]
    nc = int(m["n_cell"])
    part = P.slab_partition(m, n_parts) if method == "slab" else P.rcb_partition(m, n_parts)
    counts = np.bincount(part, minlength=n_parts)
    assert counts.sum() == nc and counts.max() - counts.min() <= n_parts
    rings = 3
    subs = P.decompose(m, part, rings)
    owner_seen = np.zeros(nc, int)
    # node adjacency on the whole grid, by brute force over the faces
    fp, fv = m["face_ptr"], m["face_vert"]
    cell_nodes = [set() for _ in range(nc)]
    for f in range(m["owner"].size):
        ns = set(fv[fp[f]:fp[f + 1]].tolist())
        cell_nodes[m["owner"][f]] |= ns
        if m["neighbour"][f] >= 0:
            cell_nodes[m["neighbour"][f]] |= ns
    for sd in subs:
        assert np.all(np.diff(sd.cells) > 0) and np.all(np.diff(sd.faces) > 0)
        assert np.all(np.diff(sd.nodes) > 0)
        owner_seen[sd.cells[sd.ring == 0]] += 1
        assert np.array_equal(np.flatnonzero(part[sd.cells] == sd.part), np.flatnonzero(sd.ring == 0))
        # ring k: shares a node with ring k-1 and with no earlier ring
        nodes_by_ring = [set().union(*(cell_nodes[c] for c in sd.cells[sd.ring == k]))
                         for k in range(rings + 1)]
        for k in range(1, rings + 1):
            for c in sd.cells[sd.ring == k]:
                assert cell_nodes[c] & nodes_by_ring[k - 1]
                if k >= 2:
                    assert not (cell_nodes[c] & nodes_by_ring[k - 2])
        # every cell within `rings` rings is there
        allc = set(sd.cells.tolist())
        for c in range(nc):
            if c not in allc:
                assert not (cell_nodes[c] & nodes_by_ring[rings - 1])
        # the sub-mesh: each local cell keeps all its faces, in grid order
        sm = sd.mesh
        assert sm["n_cell"] == sd.cells.size
        for lc in range(sd.cells.size):
            g = sd.cells[lc]
            gf = np.flatnonzero((m["owner"] == g) | (m["neighbour"] == g))
            lf = np.flatnonzero((sm["owner"] == lc) | (sm["neighbour"] == lc))
            assert np.array_equal(sd.faces[lf], gf)
        # faces between two local cells keep owner, neighbour and node order
        both = sm["neighbour"] >= 0
        gfo = sd.faces[both]
        assert np.array_equal(sd.cells[sm["owner"][both]], m["owner"][gfo])
        assert np.array_equal(sd.cells[sm["neighbour"][both]], m["neighbour"][gfo])
        for lf in np.flatnonzero(both)[:50]:
            g = sd.faces[lf]
            a = sd.nodes[sm["face_vert"][sm["face_ptr"][lf]:sm["face_ptr"][lf + 1]]]
            assert np.array_equal(a, fv[fp[g]:fp[g + 1]])
        np.testing.assert_array_equal(sm["X"], m["X"][sd.nodes])
        # exchange lists: what p receives from q is what q sends to p
        for q, idx in sd.recv.items():
            assert np.all(sd.ring[idx] > 0) and np.all(part[sd.cells[idx]] == q)
            other = subs[q]
            assert np.array_equal(other.cells[other.send[sd.part]], sd.cells[idx])
            assert np.all(other.ring[other.send[sd.part]] == 0)
        assert sum(len(v) for v in sd.recv.values()) == int((sd.ring > 0).sum())
    assert np.all(owner_seen == 1)


def test_halo_depths():
    assert P.halo_rings(P.PREC_FP64, P.RECON_LSGIR) == 3
    assert P.halo_rings(P.PREC_FP64, P.RECON_LSFIR, 4) == 7
    assert P.halo_rings(P.PREC_MIXED, P.RECON_LSGIR) == 9
    assert P.halo_rings(P.PREC_MIXED, P.RECON_LSFIR, 2) == 11


def test_partition_errors():
    m = I.hex_mesh(3)
    with pytest.raises(ValueError):
        P.slab_partition(m, 0)
    with pytest.raises(ValueError):
        P.slab_partition(m, 28)
    with pytest.raises(ValueError):
        P.decompose(m, np.zeros(5, np.int32), 3)
    with pytest.raises(ValueError):
        P.decompose(m, np.zeros(27, np.int32), 0)
    # one part: no halo, the sub-mesh is the grid
    (sd,) = P.decompose(m, np.zeros(27, np.int32), 3)
    assert sd.recv == {} and np.all(sd.ring == 0)
    assert np.array_equal(sd.mesh["face_vert"], m["face_vert"])


# ---------------------------------------------------------------- oracle steppers
class OraclePart:
    """A part stepped by the oracle (tests only): advect = faceflux + vofadv,
    reconstruct = taggrid + LSGIR/LSFIR + volume enforcement."""

    def __init__(self, sd, orc, recon):
        self.sd = sd
        self.orc = orc
        self.om = orc.Mesh(sd.mesh)
        self.recon = recon

    def set_fraction(self, F):
        self.F = np.array(F, np.float64)

    def reconstruct(self):
        self.st = self.om.reconstruct(self.F, recon=self.recon)
        self.F = self.st["F"]

    def advect(self, vel, t, dt):
        Vd, VF, _ = self.om.faceflux(vel, t, dt, self.st)
        self.F = self.om.vofadv(self.st["F"], Vd, VF)

    def gather(self, q, out):
        import torch
        out.copy_(torch.from_numpy(self.F[self.sd.send[q]]))

    def scatter(self, q, src):
        self.F[self.sd.recv[q]] = src.numpy()

    def dt_bounds(self, vel):
        return _bounds(self.om, vel)

    def owned_volume(self):
        o = self.sd.owned
        return float(np.sum(self.om.geometry()["cell_vol"][o] * self.F[o]))

    def fraction(self):
        return self.F

    def buffer(self, n):
        import torch
        return torch.empty(n, dtype=torch.float64)


def _bounds(om, vel):
    """Per axis: the smallest cell bounding-box size and the largest speed at
    a face centre of the field at t = 0 (where its time factor is 1)."""
    g = om.geometry()
    bb = g["cell_bbox"]
    h = (bb[:, 3:] - bb[:, :3]).min(axis=0)
    u = np.abs(np.array([om.velocity(vel, x, 0.0) for x in g["face_cen"]])).max(axis=0)
    return h, u


def _case(name):
    if name == "hex":
        m = I.hex_mesh(10)
        F0 = I.init_fraction(m, I.sphere((0.5, 0.45, 0.52), 0.3), levels=3)
        return m, F0, I.deformation(3.0), 0.5
    m = I.kuhn_tet_mesh(5, seed=3)
    F0 = I.init_fraction(m, I.sphere((0.5, 0.55, 0.5), 0.27), levels=3)
    return m, F0, I.rotation(2 * np.pi), 0.4


def _whole(orc, m, F0, vel, dts, recon):
    om = orc.Mesh(m)
    st = om.reconstruct(F0, recon=recon)
    out, t = [], 0.0
    for dt in dts:
        st = om.step(vel, t, dt, st, recon=recon)
        t += dt
        out.append(st["F"])
    return om, out


@pytest.mark.parametrize("name,n_parts,recon", [("hex", 2, 0), ("hex", 3, 1), ("tet", 2, 0)])
def test_partitioned_steps_equal_the_whole_grid(orc, name, n_parts, recon):
    m, F0, vel, cfl = _case(name)
    om = orc.Mesh(m)
    dts, t = [], 0.0
    for _ in range(6):
        dts.append(om.suggest_dt(vel, t, cfl, 10.0))
        t += dts[-1]
    _, whole = _whole(orc, m, F0, vel, dts, recon)
    part = P.slab_partition(m, n_parts) if n_parts == 2 else P.rcb_partition(m, n_parts)
    rings = P.halo_rings(P.PREC_FP64, recon, 4)
    pg = D.PartitionedGrid(m, part=part, rings=rings,
                           part_stepper=lambda sd: OraclePart(sd, orc, recon))
    pg.set_fraction(F0)
    pg.reconstruct()
    t = 0.0
    crossing = 0
    for k, dt in enumerate(dts):
        pg.step(vel, t, dt)
        t += dt
        F = pg.get_fraction()
        assert np.array_equal(F, whole[k]), (name, k, np.abs(F - whole[k]).max())
        # the interface crosses the partition: halo cells hold interfacial F
        for sd, pt in zip(pg.subs, pg.parts):
            h = sd.ring > 0
            crossing += int(np.sum((pt.F[h] > 0) & (pt.F[h] < 1)))
    assert crossing > 0
    # the time step from bounds reduced over the parts is the whole grid's
    b = [pt.dt_bounds(vel) for pt in pg.parts]
    hw, uw = _bounds(om, vel)
    assert np.array_equal(np.min([h for h, _ in b], axis=0), hw)
    assert np.array_equal(np.max([u for _, u in b], axis=0), uw)
    vol = pg.volume()
    ref = float(np.sum(om.geometry()["cell_vol"] * whole[-1]))
    assert abs(vol - ref) <= 1e-14 * ref


def test_one_ring_is_too_shallow(orc):
    m, F0, vel, cfl = _case("hex")
    om = orc.Mesh(m)
    dts, t = [], 0.0
    for _ in range(4):
        dts.append(om.suggest_dt(vel, t, cfl, 10.0))
        t += dts[-1]
    _, whole = _whole(orc, m, F0, vel, dts, 0)
    pg = D.PartitionedGrid(m, n_parts=2, rings=1,
                           part_stepper=lambda sd: OraclePart(sd, orc, 0))
    pg.set_fraction(F0)
    pg.reconstruct()
    t = 0.0
    diff = 0.0
    for k, dt in enumerate(dts):
        pg.step(vel, t, dt)
        t += dt
        diff = max(diff, float(np.abs(pg.get_fraction() - whole[k]).max()))
    assert diff > 1e-6


# ---------------------------------------------------------------- two gloo ranks
def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        m, F0, vel, cfl = _case("hex")
        g = D.DistributedGrid(m, lambda sd: OraclePart(sd, oracle, 0), rings=3)
        g.set_fraction(F0)
        g.reconstruct()
        hmin, umax = g.dt_bounds(vel)
        t, dts = 0.0, []
        for _ in range(5):
            # Eq. eq:cfl from the reduced bounds, written out here for the
            # deformation field (time factor cos(pi t / T))
            um = umax * abs(np.cos(np.pi * t / 3.0))
            dt = 0.5 * min(hmin[d] / um[d] for d in range(3) if um[d] > 0)
            g.step(vel, t, dt)
            t += dt
            dts.append(dt)
        cells, F = g.owned_fraction()
        vol = g.volume()
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), cells=cells, F=F, dts=np.array(dts),
                 vol=vol, hmin=hmin, umax=umax, n_recv=sum(v.size for v in g.sd.recv.values()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_step_a_partitioned_grid(tmp_path, orc):
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    world = 2
    tmp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                        join=True, start_method="spawn")
    z = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert np.array_equal(z[0]["dts"], z[1]["dts"])
    assert float(z[0]["vol"]) == float(z[1]["vol"])
    assert all(int(zz["n_recv"]) > 0 for zz in z)
    m, F0, vel, cfl = _case("hex")
    om, whole = _whole(orc, m, F0, vel, list(z[0]["dts"]), 0)
    hw, uw = _bounds(om, vel)
    assert np.array_equal(z[0]["hmin"], hw) and np.array_equal(z[0]["umax"], uw)
    F = np.full(int(m["n_cell"]), np.nan)
    for zz in z:
        assert np.all(np.isnan(F[zz["cells"]]))  # each cell owned once
        F[zz["cells"]] = zz["F"]
    assert np.array_equal(F, whole[-1])
    ref = float(np.sum(om.geometry()["cell_vol"] * whole[-1]))
    assert abs(float(z[0]["vol"]) - ref) <= 1e-14 * ref

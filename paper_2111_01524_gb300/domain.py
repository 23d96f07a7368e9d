"""A partitioned grid stepped part by part, with halo exchanges between them.

Each part of the grid (``partition.decompose``) is advanced by a stepper on
its own sub-mesh; one step is (Algorithm alg:adv, split at the exchange):

  1. every part advects (V_F of its faces, the conservative update);
  2. the halo exchange: every part gathers F over the cells it sends into a
     buffer, the buffers go to the parts that hold those cells in their halo,
     and each part scatters them into its halo cells;
  3. every part reconstructs (tags, normals, plane constants).

The time step is the grid's: each part reports its per-axis bounds of
Eq. eq:cfl, the minimum cell size and maximum speed are reduced over the
parts, and the step follows from them. The global volume is the sum over
the parts of their owned cells' volume.

``PartitionedGrid`` holds every part on one device (each part a library
context; the exchange is a device-to-device copy per pair of parts).
``DistributedGrid`` holds one part per rank of a torch.distributed group
(the exchange is a point-to-point send and receive per pair of neighbouring
ranks, the bounds and the volume are all-reduced); its stepper is any
object with the ``PartStepper`` calls, e.g. ``ContextPart``.
"""
from __future__ import annotations

import numpy as np

from . import partition as P


class ContextPart:
    """Stepper of one part on the device: a library context on the part's
    sub-mesh, with list 0 = owned cells, then one list per neighbouring part
    for the cells it receives, then one per neighbouring part for the cells
    it sends."""

    def __init__(self, sd, vof, **ctx_kw):
        self.sd = sd
        self.vof = vof
        self.ctx = vof.Context(sd.mesh, **ctx_kw)
        self.nbrs = sd.neighbours
        lists = [sd.owned]
        self.recv_list, self.send_list = {}, {}
        for q in self.nbrs:
            self.recv_list[q] = len(lists)
            lists.append(sd.recv.get(q, np.zeros(0, np.int32)))
        for q in self.nbrs:
            self.send_list[q] = len(lists)
            lists.append(sd.send.get(q, np.zeros(0, np.int32)))
        self.ctx.set_lists(lists)

    # PartStepper calls
    def set_fraction(self, F_local):
        self.ctx.set_fraction(F_local)

    def advect(self, vel, t, dt):
        self.ctx.advect(vel, t, dt)

    def reconstruct(self):
        self.ctx.reconstruct()

    def gather(self, q, out):
        self.ctx.export_list(self.send_list[q], out)

    def scatter(self, q, src):
        self.ctx.import_list(self.recv_list[q], src)

    def dt_bounds(self, vel):
        return self.ctx.dt_bounds(vel)

    def owned_volume(self):
        return self.ctx.list_volume(0)

    def fraction(self):
        return self.ctx.get_fraction()

    def buffer(self, n):
        import torch
        return torch.empty(n, dtype=torch.float64, device="cuda")


class PartitionedGrid:
    """Every part of a grid in this process: by default one library context
    each on the current device (``part_stepper``, if given, makes a part's
    stepper from its Subdomain instead).

    ``rings`` defaults to ``partition.halo_rings`` of the options; ``part``
    (one int per cell) defaults to ``n_parts`` slabs."""

    def __init__(self, mesh, n_parts=2, part=None, rings=None, part_stepper=None, **ctx_kw):
        self.n_cell = int(mesh["n_cell"])
        if part is None:
            part = P.slab_partition(mesh, n_parts)
        if rings is None:
            rings = P.halo_rings(ctx_kw.get("precision", P.PREC_FP64),
                                 ctx_kw.get("recon", P.RECON_LSGIR),
                                 ctx_kw.get("lsfir_max_iter", 0) or 4)
        self.rings = rings
        self.subs = P.decompose(mesh, part, rings)
        if part_stepper is None:
            from . import vof

            def part_stepper(sd):
                return ContextPart(sd, vof, **ctx_kw)
        self.parts = [part_stepper(sd) for sd in self.subs]
        # one buffer per (receiver, sender) pair
        self.bufs = {}
        for sd, pt in zip(self.subs, self.parts):
            for q, idx in sd.recv.items():
                self.bufs[(sd.part, q)] = pt.buffer(idx.size)

    def set_fraction(self, F):
        F = np.asarray(F, np.float64)
        for sd, pt in zip(self.subs, self.parts):
            pt.set_fraction(np.ascontiguousarray(F[sd.cells]))

    def reconstruct(self):
        for pt in self.parts:
            pt.reconstruct()

    def exchange(self):
        for (p, q), buf in self.bufs.items():
            self.parts[q].gather(p, buf)
        for (p, q), buf in self.bufs.items():
            self.parts[p].scatter(q, buf)

    def step(self, vel, t, dt):
        for pt in self.parts:
            pt.advect(vel, t, dt)
        self.exchange()
        self.reconstruct()

    def suggest_dt(self, vel, t, cfl, t_end):
        b = [pt.dt_bounds(vel) for pt in self.parts]
        hmin = np.min([h for h, _ in b], axis=0)
        umax = np.max([u for _, u in b], axis=0)
        from . import vof
        return vof.dt_from_bounds(vel, hmin, umax, t, cfl, t_end)

    def volume(self):
        return float(sum(pt.owned_volume() for pt in self.parts))

    def get_fraction(self):
        return P.assemble(self.subs, [_host(pt.fraction()) for pt in self.parts], self.n_cell)


class DistributedGrid:
    """One part per rank of a torch.distributed process group.

    ``part_stepper(sd)`` makes this rank's stepper from its Subdomain; the
    stepper provides set_fraction, advect, reconstruct, gather(q, out),
    scatter(q, src), dt_bounds(vel), owned_volume(), fraction() and
    buffer(n) (a tensor on the device its collectives use). Every rank
    builds the same partition from the same grid."""

    def __init__(self, mesh, part_stepper, rings, part=None, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n_cell = int(mesh["n_cell"])
        if part is None:
            part = P.slab_partition(mesh, self.world)
        if int(np.max(part)) + 1 != self.world:
            raise ValueError("one part per rank")
        self.subs = P.decompose(mesh, part, rings)
        self.sd = self.subs[self.rank]
        self.part = part_stepper(self.sd)
        self.recv_bufs = {q: self.part.buffer(idx.size) for q, idx in self.sd.recv.items()}
        self.send_bufs = {q: self.part.buffer(idx.size) for q, idx in self.sd.send.items()}

    def _peer(self, q):
        return q if self.group is None else self.dist.get_global_rank(self.group, q)

    def set_fraction(self, F):
        self.part.set_fraction(np.ascontiguousarray(np.asarray(F, np.float64)[self.sd.cells]))

    def reconstruct(self):
        self.part.reconstruct()

    def exchange(self):
        for q, buf in self.send_bufs.items():
            self.part.gather(q, buf)
        ops = []
        for q in self.sd.neighbours:
            if q in self.send_bufs:
                ops.append(self.dist.P2POp(self.dist.isend, self.send_bufs[q], self._peer(q),
                                           self.group))
            if q in self.recv_bufs:
                ops.append(self.dist.P2POp(self.dist.irecv, self.recv_bufs[q], self._peer(q),
                                           self.group))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        for q, buf in self.recv_bufs.items():
            self.part.scatter(q, buf)

    def step(self, vel, t, dt):
        self.part.advect(vel, t, dt)
        self.exchange()
        self.part.reconstruct()

    def dt_bounds(self, vel):
        """(hmin[3], umax[3]) reduced over the ranks."""
        import torch
        h, u = self.part.dt_bounds(vel)
        b = self.part.buffer(6)
        b.copy_(torch.as_tensor(np.concatenate([-np.asarray(h), np.asarray(u)]),
                                dtype=torch.float64))
        self.dist.all_reduce(b, op=self.dist.ReduceOp.MAX, group=self.group)
        v = b.cpu().numpy()
        return -v[:3], v[3:]

    def suggest_dt(self, vel, t, cfl, t_end):
        from . import vof
        h, u = self.dt_bounds(vel)
        return vof.dt_from_bounds(vel, h, u, t, cfl, t_end)

    def volume(self):
        import torch
        b = self.part.buffer(1)
        b.fill_(self.part.owned_volume())
        self.dist.all_reduce(b, op=self.dist.ReduceOp.SUM, group=self.group)
        return float(b.cpu()[0])

    def owned_fraction(self):
        """(grid indices, F) of this rank's owned cells."""
        o = self.sd.owned
        return self.sd.cells[o], _host(self.part.fraction())[o]


def _host(F):
    return F.cpu().numpy() if hasattr(F, "cpu") else np.asarray(F)

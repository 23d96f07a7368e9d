"""Serving loop: continuous batching of "advance this interface N steps" requests.

Each request is a grid (any mesh the library accepts), an initial volume
fraction, a prescribed velocity field and a number of time steps. The server
keeps every admitted request's mesh and state resident on the device (one
library context each, with its step captured as a CUDA graph on its own
stream), admits queued requests as soon as their estimated device memory fits
in the budget (a fraction of the GPU's free memory), issues one step per
active request per scheduling tick so that the requests' work overlaps on the
device, retires finished requests (reading their result back) and reports
arrival-to-completion latency percentiles and cell-steps/s.

The scheduling logic is independent of the GPU: ``Server`` drives a backend
object (``DeviceBackend`` here; tests use a fake one) through five calls:
``open(request)``, ``step(handle, request)``, ``pending(handle)``,
``finish(handle)`` and ``close(handle)``; a handle is a dict with the
request's step count ``k``.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    """One request: advance F0 on ``mesh`` through ``n_steps`` steps of ``vel``."""

    rid: int
    mesh: dict
    F0: np.ndarray
    vel: object
    n_steps: int
    cfl: float = 0.5
    t_end: float = 1e9
    arrival: float = 0.0           # seconds after the start of the trace
    # filled by the server
    t_admit: float = float("nan")
    t_done: float = float("nan")
    result: np.ndarray | None = None
    bytes: int = 0

    @property
    def n_cell(self):
        return int(self.mesh["n_cell"])

    @property
    def latency(self):
        return self.t_done - self.arrival


def estimate_device_bytes(mesh, precision_mixed=True):
    """Device memory of one context, from the mesh sizes (upper estimate).

    Per vertex 3 coordinates + tags + vertex->cell CSR; per face 7 geometry
    doubles, CSR, owner/neighbour, tags, V_d, V_F, rate, list; per cell
    centroid, volume, box, planes, F, tags, CSRs (faces, nodes, node
    neighbours), list. Mixed contexts add the (hi, lo) float copies.
    """
    nv = int(mesh["X"].shape[0])
    nf = int(mesh["owner"].shape[0])
    nc = int(mesh["n_cell"])
    nfv = int(mesh["face_ptr"][-1])
    nb_per_cell = 27 if mesh.get("kind") == "hex" else 100
    b = nv * (24 + 1 + 8) + nf * (56 + 8 + 8 + 1 + 24 + 4) + nfv * 4
    b += nc * (32 + 48 + 33 + 8 + 1 + 4 + 8 * 3) + nfv * 2 * 4 * 2 + nc * nb_per_cell * 4
    if precision_mixed:
        b += nv * 24 + nf * 40 + nc * (24 + 48 + 4 + 16)
    return int(b * 1.1) + (1 << 20)


class DeviceBackend:
    """Runs requests on the GPU through the library's C-ABI."""

    def __init__(self, precision_mixed=True, use_graphs=True):
        import torch
        from . import vof
        self.torch = torch
        self.vof = vof
        self.prec = vof.PREC_MIXED if precision_mixed else vof.PREC_FP64
        self.use_graphs = use_graphs

    def free_bytes(self):
        free, _total = self.torch.cuda.mem_get_info()
        return int(free)

    def open(self, req):
        torch = self.torch
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = self.vof.Context(req.mesh, precision=self.prec)
            ctx.set_fraction(req.F0)  # host buffer: synchronises the stream
            ctx.reconstruct()
            if self.use_graphs:
                ctx.graph_capture(with_reconstruct=True)
        return {"ctx": ctx, "stream": stream, "events": [], "t": 0.0, "k": 0}

    def step(self, h, req):
        """Queue one time step of the request on its stream."""
        torch = self.torch
        ctx, s = h["ctx"], h["stream"]
        with torch.cuda.stream(s):
            dt = ctx.suggest_dt(req.vel, h["t"], req.cfl, req.t_end)
            if self.use_graphs:
                ctx.graph_launch([req.vel], [h["t"]], [dt])
            else:
                ctx.step(req.vel, h["t"], dt)
            ev = torch.cuda.Event()
            ev.record(s)
        h["events"].append(ev)
        h["t"] += dt
        h["k"] += 1

    def pending(self, h):
        """Steps of the request still running on the device."""
        ev = h["events"]
        while ev and ev[0].query():
            ev.pop(0)
        return len(ev)

    def finish(self, h):
        torch = self.torch
        with torch.cuda.stream(h["stream"]):
            F = h["ctx"].get_fraction()  # synchronises the request's stream
        return F

    def close(self, h):
        h["ctx"].close()


@dataclass
class ServeStats:
    latencies: list = field(default_factory=list)
    cell_steps: int = 0
    wall: float = 0.0
    admitted: int = 0
    max_active: int = 0
    max_bytes: int = 0

    def summary(self):
        lat = np.asarray(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "cell_steps_per_s": self.cell_steps / self.wall if self.wall > 0 else 0.0,
                "wall_s": self.wall, "max_active": self.max_active,
                "max_resident_bytes": self.max_bytes}


class Server:
    """Continuous-batching scheduler over a backend.

    ``budget_bytes``: device memory the resident requests may use in total
    (default: ``budget_fraction`` of the backend's free memory at start).
    ``max_inflight``: steps a request may have queued on the device before
    the scheduler waits for it (bounds the host running ahead).
    """

    def __init__(self, backend, budget_bytes=None, budget_fraction=0.8, max_active=256,
                 max_inflight=2, clock=time.perf_counter, sleep=time.sleep):
        self.backend = backend
        if budget_bytes is None:
            budget_bytes = int(budget_fraction * backend.free_bytes())
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.max_inflight = max_inflight
        self.clock = clock
        self.sleep = sleep

    def run(self, requests, estimate=estimate_device_bytes):
        """Serve the requests (each with its ``arrival`` offset) to completion."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            r.bytes = int(estimate(r.mesh))
            if r.bytes > self.budget:
                raise ValueError(f"request {r.rid} needs {r.bytes} bytes, over the budget "
                                 f"{self.budget}")
        queue = []          # arrived, not admitted (FIFO by arrival)
        active = {}         # rid -> (request, handle)
        resident = 0
        stats = ServeStats()
        t0 = self.clock()
        i = 0
        while i < len(pending) or queue or active:
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                heapq.heappush(queue, (pending[i].arrival, pending[i].rid, pending[i]))
                i += 1
            # admission by memory budget, in arrival order
            while queue and len(active) < self.max_active and resident + queue[0][2].bytes <= self.budget:
                _, _, r = heapq.heappop(queue)
                r.t_admit = self.clock() - t0
                active[r.rid] = (r, self.backend.open(r))
                resident += r.bytes
                stats.admitted += 1
            stats.max_active = max(stats.max_active, len(active))
            stats.max_bytes = max(stats.max_bytes, resident)
            # one more step for every active request with room in flight;
            # retire the requests whose last step has completed
            progressed = False
            for rid in list(active):
                r, h = active[rid]
                inflight = self.backend.pending(h)
                if h["k"] >= r.n_steps:
                    if inflight == 0:
                        r.result = self.backend.finish(h)
                        r.t_done = self.clock() - t0
                        self.backend.close(h)
                        del active[rid]
                        resident -= r.bytes
                        stats.latencies.append(r.latency)
                        stats.cell_steps += r.n_cell * r.n_steps
                        progressed = True
                    continue
                if inflight < self.max_inflight:
                    self.backend.step(h, r)
                    progressed = True
            if not progressed:
                if not active and not queue and i < len(pending):
                    self.sleep(max(0.0, min(0.01, pending[i].arrival - (self.clock() - t0))))
                else:
                    self.sleep(0.0002)
        stats.wall = self.clock() - t0
        return stats


def poisson_trace(n, rate, seed, make_request):
    """n requests with exponential inter-arrival times of mean 1/rate;
    ``make_request(rid, rng)`` builds request rid."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        t += rng.exponential(1.0 / rate)
        r = make_request(rid, rng)
        r.arrival = t
        out.append(r)
    return out

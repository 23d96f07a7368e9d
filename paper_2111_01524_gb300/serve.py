"""Replay of a request trace through the device-resident serving loop.

A request is "advance this interface N steps": a grid (any mesh the library
accepts), an initial volume fraction, a prescribed velocity field, a number
of time steps and a CFL number. The serving loop itself is the library's
``vof_server_*`` (continuous batching: requests are admitted within a device
memory budget as the slots of batched contexts, and every live context
advances one step per scheduling tick; see ``include/vof.h``). This module
only submits the requests of a trace at their arrival times, ticks the
server and collects the results; the server object may be ``vof.Server`` or
any object with the same ``submit`` / ``step`` / ``poll`` calls (the tests
use a simulated one).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


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
    # filled by replay()
    sid: int = -1
    t_submit: float = float("nan")
    t_done: float = float("nan")
    latency: float = float("nan")  # arrival (= submission) to result, server clock
    result: np.ndarray | None = None

    @property
    def n_cell(self):
        return int(self.mesh["n_cell"])


@dataclass
class ReplayStats:
    latencies: list = field(default_factory=list)
    cell_steps: int = 0
    wall: float = 0.0
    ticks: int = 0
    max_active: int = 0

    def summary(self):
        lat = np.asarray(self.latencies) if self.latencies else np.zeros(1)
        return {"requests": len(self.latencies), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "cell_steps_per_s": self.cell_steps / self.wall if self.wall > 0 else 0.0,
                "wall_s": self.wall, "ticks": self.ticks, "max_active": self.max_active}


def replay(server, requests, clock=time.perf_counter, sleep=time.sleep):
    """Submit each request when its ``arrival`` offset has passed, tick the
    server until every request is done, and collect results and latencies."""
    pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
    live = {}
    stats = ReplayStats()
    t0 = clock()
    i = 0
    while i < len(pending) or live:
        now = clock() - t0
        while i < len(pending) and pending[i].arrival <= now:
            r = pending[i]
            r.t_submit = now
            r.sid = server.submit(r.mesh, r.F0, r.vel, r.n_steps, r.cfl, r.t_end)
            live[r.sid] = r
            i += 1
        n_active = server.step() if live else 0
        stats.ticks += 1 if live else 0
        stats.max_active = max(stats.max_active, n_active)
        for sid in list(live):
            state, F, lat = server.poll(sid)
            if state == REQ_DONE:
                r = live.pop(sid)
                r.result = F
                r.t_done = clock() - t0
                r.latency = lat
                stats.latencies.append(lat)
                stats.cell_steps += r.n_cell * r.n_steps
        if not live and i < len(pending):
            sleep(max(0.0, min(0.01, pending[i].arrival - (clock() - t0))))
        elif live and n_active == 0:
            sleep(0.0002)  # only queued requests or result copies in flight
    stats.wall = clock() - t0
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

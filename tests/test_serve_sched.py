"""Host logic of the trace replay on CPU with a simulated server: requests
are submitted at their arrival times, the server is ticked while requests
are pending, every result is collected once with its latency, and the trace
generator is deterministic. (The device-resident scheduler itself, its
admission by budget and its batching, runs in the library and is tested on
the GPU in tests/test_gpu_server.py.)"""
import numpy as np

from paper_2111_01524_gb300 import serve


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-4)


class SimServer:
    """Admits every submitted request at the next tick; each tick advances
    every admitted request one step and takes `tick_s` of simulated time; a
    request is done one tick after its last step (the result copy)."""

    def __init__(self, clock, tick_s=0.001):
        self.clock = clock
        self.tick_s = tick_s
        self.reqs = []
        self.submit_log = []

    def submit(self, mesh, F0, vel, n_steps, cfl, t_end):
        sid = len(self.reqs)
        self.reqs.append({"k": -1, "n": n_steps, "F": np.array(F0, float), "t0": self.clock(),
                          "done": None, "cfl": cfl})
        self.submit_log.append((self.clock(), sid))
        return sid

    def step(self):
        n = 0
        for r in self.reqs:
            if r["done"] is not None:
                continue
            if r["k"] < 0:
                r["k"] = 0
            elif r["k"] < r["n"]:
                r["k"] += 1
                r["F"] = np.clip(0.5 * (r["F"] + np.roll(r["F"], 1)) + 1e-3 * r["k"], 0, 1)
                n += 1
            else:
                r["done"] = self.clock() + self.tick_s
        self.clock.t += self.tick_s
        return n

    def poll(self, sid):
        r = self.reqs[sid]
        if r["done"] is not None and r["done"] <= self.clock():
            return serve.REQ_DONE, r["F"].copy(), r["done"] - r["t0"]
        return serve.REQ_RUNNING, None, -1.0


def _req(rid, n_cells, steps, arrival):
    mesh = {"n_cell": n_cells}
    return serve.Request(rid=rid, mesh=mesh, F0=np.linspace(0, 1, n_cells), vel=None,
                         n_steps=steps, arrival=arrival)


def test_requests_are_submitted_at_their_arrival_and_all_finish():
    clock = SimClock()
    srv = SimServer(clock)
    reqs = [_req(0, 5, 4, 0.0), _req(1, 7, 2, 0.05), _req(2, 3, 6, 0.0021)]
    st = serve.replay(srv, reqs, clock=clock, sleep=clock.sleep)
    # submitted in arrival order, none before its arrival
    order = [sid for _, sid in srv.submit_log]
    assert [reqs[0].sid, reqs[2].sid, reqs[1].sid] == order
    for r in reqs:
        assert r.t_submit >= r.arrival
        assert r.result is not None and r.t_done >= r.t_submit
        assert r.latency > 0
    assert st.cell_steps == 5 * 4 + 7 * 2 + 3 * 6
    assert len(st.latencies) == 3 and st.max_active >= 2
    assert st.summary()["requests"] == 3


def test_results_do_not_depend_on_the_other_requests():
    """The simulated result of a request is a function of the request only:
    replayed alone or in a mix it is the same."""
    def run(reqs):
        clock = SimClock()
        serve.replay(SimServer(clock), reqs, clock=clock, sleep=clock.sleep)
        return {r.rid: r.result for r in reqs}
    mix = run([_req(i, 4 + i, 2 + i, 0.003 * i) for i in range(6)])
    for i in range(6):
        alone = run([_req(i, 4 + i, 2 + i, 0.0)])
        assert np.array_equal(alone[i], mix[i])


def test_poisson_trace_is_deterministic():
    def mk(rid, rng):
        return _req(rid, 10, int(rng.integers(1, 5)), 0.0)
    a = serve.poisson_trace(20, 200.0, 7, mk)
    b = serve.poisson_trace(20, 200.0, 7, mk)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert [r.n_steps for r in a] == [r.n_steps for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert (gaps > 0).all() and abs(gaps.mean() - 1 / 200.0) < 3 / 200.0

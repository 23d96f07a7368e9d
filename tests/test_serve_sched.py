"""Host logic of the serving loop on CPU with a simulated device:
admission by memory budget, FIFO order, overlap, completion and latency."""
import numpy as np
import pytest

from paper_2111_01524_gb300 import serve


class SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-4)


class FakeBackend:
    """Each step takes `step_s` of simulated device time per request; requests
    run concurrently (separate streams)."""

    def __init__(self, clock, step_s=0.01):
        self.clock = clock
        self.step_s = step_s
        self.open_log = []
        self.live = set()
        self.peak_live = 0

    def free_bytes(self):
        return 10 ** 9

    def open(self, r):
        self.open_log.append((self.clock(), r.rid))
        self.live.add(r.rid)
        self.peak_live = max(self.peak_live, len(self.live))
        return {"rid": r.rid, "k": 0, "busy_until": self.clock(), "steps": []}

    def step(self, h, r):
        start = max(self.clock(), h["busy_until"])
        h["busy_until"] = start + self.step_s
        h["steps"].append(h["busy_until"])
        h["k"] += 1
        self.clock.t += 1e-5  # host cost of issuing

    def pending(self, h):
        h["steps"] = [t for t in h["steps"] if t > self.clock()]
        return len(h["steps"])

    def finish(self, h):
        return np.full(3, float(h["rid"]))

    def close(self, h):
        self.live.discard(h["rid"])


def _req(rid, n_cells, steps, arrival):
    mesh = {"n_cell": n_cells, "X": np.zeros((1, 3)), "owner": np.zeros(1, np.int32),
            "face_ptr": np.zeros(2, np.int64)}
    return serve.Request(rid=rid, mesh=mesh, F0=np.zeros(n_cells), vel=None, n_steps=steps,
                         arrival=arrival)


def test_budget_admission_and_completion():
    clock = SimClock()
    be = FakeBackend(clock)
    reqs = [_req(i, 100, 5, 0.001 * i) for i in range(6)]
    # every request "needs" 40 bytes; the budget fits two at a time
    srv = serve.Server(be, budget_bytes=80, clock=clock, sleep=clock.sleep)
    st = srv.run(reqs, estimate=lambda m: 40)
    assert len(st.latencies) == 6
    assert st.max_bytes <= 80 and st.max_active == 2 and be.peak_live == 2
    # admitted in arrival order
    assert [rid for _, rid in be.open_log] == list(range(6))
    for r in reqs:
        assert r.t_admit >= r.arrival and r.t_done > r.t_admit
        assert np.all(r.result == r.rid)
    assert st.cell_steps == 6 * 100 * 5


def test_requests_overlap_when_budget_allows():
    clock = SimClock()
    be = FakeBackend(clock, step_s=0.01)
    reqs = [_req(i, 10, 10, 0.0) for i in range(8)]
    srv = serve.Server(be, budget_bytes=10 ** 6, clock=clock, sleep=clock.sleep)
    st = srv.run(reqs, estimate=lambda m: 10)
    # 8 concurrent requests of 10 steps x 10 ms finish in about 100 ms, not 800
    assert st.wall < 0.2 and be.peak_live == 8


def test_oversized_request_is_rejected():
    clock = SimClock()
    srv = serve.Server(FakeBackend(clock), budget_bytes=10, clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.run([_req(0, 10, 1, 0.0)], estimate=lambda m: 11)


def test_poisson_trace_is_seeded_and_sorted():
    mk = lambda rid, rng: _req(rid, 1, 1, 0.0)
    a = serve.poisson_trace(20, 200.0, 7, mk)
    b = serve.poisson_trace(20, 200.0, 7, mk)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert 0.05 < a[-1].arrival < 0.2

"""Multi-rank path on CPU: the grids of a batch and the requests of a stream
are sharded across ranks by estimated work with no data-path collective.

Two gloo ranks (world size 2, rendezvous on 127.0.0.1) each compute the
partition on their own, serve their share through the serving loop with a
simulated device, and report the bookkeeping the benchmark does over ranks
(barrier, slowest rank's time, total cell-steps). The union of the shares
must be every unit exactly once, the partition must agree between ranks, and
every result must equal the one a single rank computes.
"""
import os
import socket

import numpy as np
import pytest

from paper_2111_01524_gb300 import serve, shard


# ---------------------------------------------------------------- partition
def test_balance_covers_every_unit_once_and_is_deterministic():
    rng = np.random.default_rng(3)
    w = rng.integers(1, 10 ** 6, 97).astype(float)
    for world in (1, 2, 3, 8):
        parts = shard.balance(w, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(w)))
        assert parts == shard.balance(w, world)
        # LPT bound: no rank exceeds the mean load by more than the largest unit
        ld = shard.loads(w, parts)
        assert max(ld) <= w.sum() / world + w.max() + 1e-9


def test_balance_edge_cases():
    assert shard.balance([], 2) == [[], []]
    assert shard.balance([5.0], 3) == [[0], [], []]
    # equal weights: round robin in index order
    assert shard.balance([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.balance([1.0], 0)
    with pytest.raises(ValueError):
        shard.balance([1.0, -1.0], 2)


# ---------------------------------------------------------------- two gloo ranks
class _SimClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, d):
        self.t += max(d, 1e-4)


class _SimServer:
    """A stand-in for the device-resident server (the GPU is not needed for
    the host logic): every submitted request is admitted at the next tick
    and advanced one step per tick; its result is a fixed map of its own F0
    and step count, so it must not depend on which rank serves it."""

    def __init__(self, clock, tick_s=0.001):
        self.clock = clock
        self.tick_s = tick_s
        self.reqs = []

    def submit(self, mesh, F0, vel, n_steps, cfl, t_end):
        self.reqs.append({"k": -1, "n": n_steps, "F": np.array(F0, float), "t0": self.clock(),
                          "done": None})
        return len(self.reqs) - 1

    def step(self):
        n = 0
        for r in self.reqs:
            if r["done"] is not None:
                continue
            if r["k"] < 0:
                r["k"] = 0
            elif r["k"] < r["n"]:
                r["k"] += 1
                r["F"] = np.clip(0.5 * (r["F"] + np.roll(r["F"], 1)) + 1e-3 * r["k"], 0.0, 1.0)
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


def _requests():
    rng = np.random.default_rng(11)
    out = []
    for rid in range(23):
        n = int(rng.integers(50, 400))
        mesh = {"n_cell": n}
        out.append(serve.Request(rid=rid, mesh=mesh, F0=rng.random(n), vel=None,
                                 n_steps=int(rng.integers(3, 12)), arrival=0.002 * rid))
    return out


def _serve(reqs):
    clock = _SimClock()
    st = serve.replay(_SimServer(clock), reqs, clock=clock, sleep=clock.sleep)
    return st, {r.rid: r.result for r in reqs}


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        reqs = _requests()
        weights = [r.n_cell * r.n_steps for r in reqs]
        parts = shard.balance(weights, world)
        mine = [reqs[i] for i in parts[rank]]
        dist.barrier()
        st, results = _serve(mine)
        dist.barrier()
        # the benchmark's bookkeeping: slowest rank's time, total cell-steps
        t = torch.tensor([st.wall], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        cs = torch.tensor([st.cell_steps], dtype=torch.float64)
        dist.all_reduce(cs, op=dist.ReduceOp.SUM)
        # every rank's partition must be the same
        flat = torch.tensor([i for p in parts for i in p] + [-1] + [len(p) for p in parts])
        gathered = [torch.zeros_like(flat) for _ in range(world)]
        dist.all_gather(gathered, flat)
        same = all(bool(torch.equal(g, flat)) for g in gathered)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"),
                 rids=np.array(sorted(results)), wall=st.wall, max_wall=float(t.item()),
                 total_cs=float(cs.item()), own_cs=float(st.cell_steps), same=same,
                 **{f"F{rid}": F for rid, F in results.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_the_stream(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    world = 2
    tmp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                        join=True, start_method="spawn")
    single_st, single = _serve(_requests())
    got = {}
    walls = []
    for rank in range(world):
        z = np.load(tmp_path / f"rank{rank}.npz")
        assert bool(z["same"])
        walls.append(float(z["wall"]))
        assert float(z["total_cs"]) == single_st.cell_steps
        for rid in z["rids"]:
            assert int(rid) not in got  # no unit served twice
            got[int(rid)] = z[f"F{int(rid)}"]
    assert sorted(got) == sorted(single)
    for rid, F in single.items():
        assert np.array_equal(got[rid], F), rid
    for rank in range(world):
        assert float(np.load(tmp_path / f"rank{rank}.npz")["max_wall"]) == max(walls)

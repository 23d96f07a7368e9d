#!/usr/bin/env python
"""Benchmark of the unsplit geometric VOF hot path (LSGIR + FMFPA) on GB300.

Metric: VOF cell-steps/s over reconstruct + advect (the paper's
t_cpu = t_rec + t_adv), on the 3D deformation test (Sec. 4.2.3): uniform
hexahedral grid on the unit cube, sphere r = 0.15 at (0.35, 0.35, 0.35),
period T = 3, CFL 0.5, time steps from Eq. eq:cfl. Default grid 256^3
(16.8 M cells), mixed precision (FP32 geometry, FP64 roots near F = 0/1,
updates and sums) with the plain FP64 path measured beside it.

A step is one iteration of the advection loop: faceflux + vofadv + taggrid +
LSGIR + plane constant, i.e. every kernel of the hot path. Inputs (mesh,
F, planes) are resident in HBM and far larger than L2 (the mesh arrays
alone are ~10 GB at 256^3), so no L2 flush is needed between steps.

Multi-GPU (no data-path collective anywhere): the single-grid workloads run
one independent replica per rank; the batched and served workloads shard
their independent units (grids, requests) across ranks by estimated work
(cells x steps). value = total cell-steps of all ranks / the slowest rank's
time.

--impl reference times the FP64 CPU oracle (test infrastructure) on the
host cores on the same workload, one full step per timed step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2111_01524_gb300 import inputs as I  # noqa: E402

METRIC = "VOF cell-steps/s (recon+advect) mixed vs FP64 at stated F error; p50/p99 latency"
UNIT = "cell-steps/s"
# algorithmic work per unit of the band kernels: flops of one flux-polyhedron
# construction (k_prebuild, per active face) and of one (face, cell)
# truncation with its divergence sum (k_flux)
FLOPS_PER_ACTIVE_FACE = 350.0      # FMFPA construction
FLOPS_PER_TRUNCATION = 1200.0      # one (face, cell) truncation incl. volume
# EMFPA (Sec. 2.2.1): one velocity per vertex instead of two but five
# triangle volumes per vertex; its surface has twice the face-vertex loop
# entries of FMFPA (64 against 32 for a hex face), and a truncation's
# clipping and divergence sum scale with those entries
# NMFPA (Sec. 2.2.3): one velocity per face and a translation; its prism has
# 6I loop entries (24 for a hex face, against 32)
FLOPS = {"fmfpa": (FLOPS_PER_ACTIVE_FACE, FLOPS_PER_TRUNCATION), "emfpa": (400.0, 2400.0),
         "nmfpa": (100.0, 900.0)}
# ncu --set full of the mixed flux kernel (128^3 deformation, 4th step's launch, ~57,400
# active faces) per flux-polyhedron construction: dram__bytes_read.sum +
# dram__bytes_write.sum per active face (the face and node data, the prebuilt
# polyhedron, the candidate cells' tags, boxes and planes), issue-slot and FMA-pipe
# use; valid only for the source it was taken on (traffic is null for any other)
# ncu figures of k_flux per flux polyhedron (one launch, --set full), valid
# for the k_flux.cu source whose sha256 they carry
FLUX_NCU = {"fmfpa": {"source_sha256": "cc7141663a57a88a91845e222e8372ba1d47e60e63fad7ad505f10462c452892",
                      "dram_bytes_per_active_face": 586.0, "issue_active": 0.674,
                      "fma_pipe_active": 0.176,
                      "capture": "profiles/k_flux_deformation128_midrun_mixed.md"},
            "emfpa": {"source_sha256": "f73470b1044dd746c14f9f88973f6e28d1146cc8accd65f66cc0f6bb326d8456",
                      "dram_bytes_per_active_face": 590.0, "issue_active": 0.573,
                      "fma_pipe_active": 0.149,
                      "capture": "profiles/k_flux_deformation128_mixed_emfpa.md"},
            "nmfpa": {"source_sha256": "f73470b1044dd746c14f9f88973f6e28d1146cc8accd65f66cc0f6bb326d8456",
                      "dram_bytes_per_active_face": 566.0, "issue_active": 0.528,
                      "fma_pipe_active": 0.136,
                      "capture": "profiles/k_flux_deformation128_mixed_nmfpa.md"}}
# kernels one step launches: reconstruction (cell tags 1, node tags 3,
# LSGIR 1, in mixed precision 2, or LSFIR 1 + 2 n_out) and advection (face sweep 2, polyhedra 1,
# flux 1, update 2, and in mixed precision the candidate lists of the
# prebuilt polyhedra 1 and the reconciliation of FP32 noise: 5 per round x 3
# rounds + 1); the phase timers count the same kernels
REPAIR_LAUNCHES = 5 * 3 + 1


def recon_kernels(recon="lsgir", n_out=4, precision="mixed"):
    # LSGIR: the warp kernel, and in the mixed path the closed form of the
    # box cells' plane constants
    return 4 + (1 + 2 * n_out if recon == "lsfir" else (2 if precision == "mixed" else 1))


def advect_kernels(precision="mixed", prebuilt=True):
    # the mixed path with prebuilt polyhedra also lists their candidate cells
    return 6 + ((1 if prebuilt else 0) + REPAIR_LAUNCHES if precision == "mixed" else 0)


def kernels_per_step(recon="lsgir", n_out=4, precision="mixed", prebuilt=True):
    return recon_kernels(recon, n_out, precision) + advect_kernels(precision, prebuilt)


FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2
N_SM = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gvof", choices=["gvof", "reference"])
    p.add_argument("--grid", type=int, default=256)
    p.add_argument("--grid2d", type=int, default=1024, help="n of the n x 1 x n 2D grid")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--flux", default="fmfpa", choices=["fmfpa", "emfpa", "nmfpa"],
                   help="flux polyhedron: face-matched (Sec. 2.2.2), edge-matched (Sec. 2.2.1) "
                        "or non-matched (Sec. 2.2.3)")
    p.add_argument("--recon", default="lsgir", choices=["lsgir", "lsfir"],
                   help="interface reconstruction: LSGIR (Sec. 2.1.1) or LSFIR (Sec. 2.1.2)")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-init", action="store_true", help="skip timing the device initialisation")
    p.add_argument("--cpu-steps", type=int, default=1)
    p.add_argument("--workload", default="deformation",
                   choices=["deformation", "tets", "batch", "serve", "deform2d", "cycle128"],
                   help="deformation: hex grid, Enright field (default line); tets: jittered Kuhn "
                        "tets in rotation; batch: 64 distorted grids advanced together; serve: "
                        "Poisson request stream; deform2d: 2D deformation on a quasi-2D grid; "
                        "cycle128: the whole 128^3 run of the oracle beside both GPU paths")
    p.add_argument("--requests", type=int, default=256)
    p.add_argument("--budget-frac", type=float, default=0.8,
                   help="serving: device budget as a fraction of the free memory")
    p.add_argument("--max-batch", type=int, default=16,
                   help="serving: requests admitted into one batched context per tick")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(grid):
    mesh = I.hex_mesh(grid)
    F0 = I.init_fraction(mesh, I.sphere((0.35, 0.35, 0.35), 0.15), levels=4)
    return mesh, F0, I.deformation(3.0), 0.5, 3.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init():
    """One rank per GPU; the process group carries only the barrier and the
    measurement bookkeeping."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local, dist


def over_ranks(dist, value, op):
    """max / sum of a host float over ranks (identity on one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def run_steps(ctx, vel, cfl, t_end, t, n, stream, timing=False):
    """n steps of the advection loop; returns new t and per-step ms (events)."""
    import torch
    evs = []
    for _ in range(n):
        dt = ctx.suggest_dt(vel, t, cfl, t_end)
        if timing:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        ctx.step(vel, t, dt, stream=stream)
        if timing:
            e1.record(stream)
            evs.append((e0, e1))
        t += dt
    return t, evs


def roofline(ctx_counts, phase, grid_counts, peaks, peak_kind, clocks, precision, flux="fmfpa",
             oflops=None):
    """Roofline of the dominant phase's main kernel: algorithmic HBM bytes per
    launch for the sweeps, algorithmic flops per launch for the band kernels.
    Each phase runs once per step; the flux phase is the one k_flux launch.
    oflops: the oracle's op count for the truncations of the same state's
    active faces (flops per active face), which replaces the estimate."""
    ms, calls = phase["ms"], phase["calls"]
    per_launch_ms = ms / max(calls, 1)
    nc, nf, nv = grid_counts["n_cell"], grid_counts["n_face"], grid_counts["n_vert"]
    name = phase["name"]
    hbm_bytes = {
        "cell_tags": nc * (8 + 1),
        "node_tags": nv * (8 + 1) + 8 * nc * 4 + nc * 8,
        "face_sweep": nf * (8 + 16 + 1) + nv,
        "update": nc * (8 + 24 + 16 + 8) + nf * (8 + 1),
    }
    if name in hbm_bytes:
        b = hbm_bytes[name]
        achieved = b / (per_launch_ms * 1e-3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "algorithmic_bytes_per_launch": b, "peak_source": peak_kind}
    # band kernels: plain ALU arithmetic
    # the counters describe the last advect (one launch of each band kernel);
    # the flux kernel truncates polyhedra built by the polyhedra phase
    f_face, f_trunc = FLOPS[flux]
    flops_src = "estimate"
    if name == "polyhedra":
        fl = ctx_counts["n_active_faces"] * f_face
    elif oflops is not None:
        fl = ctx_counts["n_active_faces"] * oflops["flops_per_active_face"]
        flops_src = ("oracle op counter: the FP64 oracle's arithmetic for the truncations of the "
               "same state's active faces (tetrahedral decomposition, "
               f"{oflops['flops_per_truncation']:.0f} flops per truncation), per active face "
               "x this launch's active faces")
    else:
        fl = ctx_counts["n_truncations"] * f_trunc
    traffic, ncu = None, None
    if name == "flux" and precision == "mixed":
        import hashlib
        src = os.path.join(ROOT, "paper_2111_01524_gb300", "csrc", "k_flux.cu")
        rec = FLUX_NCU.get(flux)  # the capture's figures, if it was taken on this source
        if rec is not None and hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
            rec = None
        if rec is not None:
            traffic = rec["dram_bytes_per_active_face"] * ctx_counts["n_active_faces"]
            ncu = {k: rec[k] for k in ("issue_active", "fma_pipe_active", "capture")}
    mhz = clocks.get("sm_mhz") or 1900.0
    lanes = FP32_LANES_PER_SM if precision == "mixed" else FP64_LANES_PER_SM
    peak = N_SM * lanes * 2 * mhz * 1e6 / 1e12
    achieved = fl / (per_launch_ms * 1e-3) / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "ncu": ncu,
            "algorithmic_flops_per_launch": fl, "flops_source": flops_src,
            "peak_source": f"{'FP32' if precision == 'mixed' else 'FP64'} FMA lanes x SMs x "
                           f"median SM clock {mhz:.0f} MHz"}


def cpu_baseline(mesh, F0, vel, cfl, t_end, steps, flux="fmfpa", recon="lsgir"):
    import oracle
    oracle.build()
    om = oracle.Mesh(mesh)
    st = om.reconstruct(F0)
    t = 0.0
    t0 = time.perf_counter()
    method = {"emfpa": oracle.EMFPA, "nmfpa": oracle.NMFPA}.get(flux, oracle.FMFPA)
    rc = oracle.LSFIR if recon == "lsfir" else oracle.LSGIR
    if rc == oracle.LSFIR:
        st = om.reconstruct(F0, recon=rc)
    for _ in range(steps):
        dt = om.suggest_dt(vel, t, cfl, t_end)
        st = om.step(vel, t, dt, st, method=method, recon=rc)
        t += dt
    el = time.perf_counter() - t0
    return {"value": om.n_cell * steps / el, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} full step(s) of the {round(om.n_cell ** (1 / 3))}^3 workload "
                      f"from t=0 (FP64 C oracle, OpenMP; mesh build excluded)"}


def midcycle_state(a, mesh, F0, vel, cfl, t_end):
    """F at the first warm-up step of the default line's timed segment, and
    the segment's time levels: the run from t = 0 is advanced to there with
    the library (mixed precision) when a GPU is present; it prepares the
    input of the oracle's timed steps and is not timed."""
    import torch
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    ctx = V.Context(mesh, precision=V.PREC_MIXED)
    ctx.set_fraction(torch.from_numpy(F0).cuda())
    ctx.reconstruct()
    levels = cycle_levels(ctx, vel, cfl, t_end)
    N = len(levels)
    s0 = max(a.warmup, N // 2 - a.steps // 2)
    for t, dt in levels[:s0 - a.warmup]:
        ctx.step(vel, t, dt)
    F = ctx.get_fraction()
    del ctx
    torch.cuda.empty_cache()
    return F, levels[s0 - a.warmup:s0 + a.steps], N, s0


def main_reference(a):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    mesh, F0, vel, cfl, t_end = workload(a.grid)
    counts = I.mesh_counts(mesh)
    F, seg, N, s0 = midcycle_state(a, mesh, F0, vel, cfl, t_end)
    import oracle
    oracle.build()
    om = oracle.Mesh(mesh)
    method = {"emfpa": oracle.EMFPA, "nmfpa": oracle.NMFPA}.get(a.flux, oracle.FMFPA)
    rc = oracle.LSFIR if a.recon == "lsfir" else oracle.LSGIR
    st = om.reconstruct(F, recon=rc)
    for t, dt in seg[:a.warmup]:
        st = om.step(vel, t, dt, st, method=method, recon=rc)
    lat = []
    t0 = time.perf_counter()
    for t, dt in seg[a.warmup:]:
        s_ = time.perf_counter()
        st = om.step(vel, t, dt, st, method=method, recon=rc)
        lat.append((time.perf_counter() - s_) * 1e3)
    el = time.perf_counter() - t0
    value = om.n_cell * a.steps / el
    sample = (f"{a.steps} full oracle steps (after {a.warmup} untimed) of the segment: the state "
              f"at step {s0 - a.warmup} of the {N}-step run was prepared by the library (mixed "
              f"precision, not timed), then only the FP64 C oracle (OpenMP) runs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": el * 1e3 / a.steps,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": segment_config(a, counts, N, s0),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main_cycle(a):
    """The hex deformation at 128^3 to t = 3: the oracle's whole run (multi-core) beside
    the mixed and FP64 GPU paths; end-of-run shape error (Sec. 4.2, E_shape
    against the initial shape, which the field returns to at t = T) and the
    volume of each, and the mixed path's F against the oracle's."""
    import torch
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    grid = 128 if a.grid == 256 else a.grid
    mesh, F0, vel, cfl, t_end = workload(grid)
    res = {}
    Vc = None
    for name, prec in (("mixed", V.PREC_MIXED), ("fp64", V.PREC_FP64)):
        ctx = V.Context(mesh, precision=prec)
        ctx.set_fraction(torch.from_numpy(F0).cuda())
        ctx.reconstruct()
        levels = cycle_levels(ctx, vel, cfl, t_end)
        Vc = ctx.geometry()["cell_vol"]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for t, dt in levels:
            ctx.step(vel, t, dt)
        e1.record()
        torch.cuda.synchronize()
        F = ctx.get_fraction()
        s = ctx.stats()
        res[name] = {"F": F, "ms": e0.elapsed_time(e1), "steps": len(levels), "stats": s}
        del ctx
    import oracle
    oracle.build()
    om = oracle.Mesh(mesh)
    st = om.reconstruct(F0)
    t0 = time.perf_counter()
    for t, dt in levels:
        st = om.step(vel, t, dt, st)
    el = time.perf_counter() - t0
    Fo = st["F"]
    vol0 = float((Vc * F0).sum())
    out = {"workload": f"3D deformation, hex {grid}^3, sphere r=0.15, T=3, CFL 0.5, whole run",
           "steps": len(levels), "oracle": {"s": el, "cores": oracle.num_threads(),
                                            "cell_steps_per_s": om.n_cell * len(levels) / el,
                                            "e_shape": float((Vc * np.abs(Fo - F0)).sum()),
                                            "volume_rel_change": float((Vc * Fo).sum() / vol0 - 1)}}
    for name, r in res.items():
        F = r["F"]
        out[name] = {"ms": r["ms"], "cell_steps_per_s": om.n_cell * r["steps"] / (r["ms"] * 1e-3),
                     "e_shape": float((Vc * np.abs(F - F0)).sum()),
                     "volume_rel_change": float((Vc * F).sum() / vol0 - 1),
                     "volume_rel_diff_vs_oracle": float(abs((Vc * F).sum() - (Vc * Fo).sum()) / vol0),
                     "max_abs_F_diff_vs_oracle": float(np.abs(F - Fo).max()),
                     "l1_rel_F_diff_vs_oracle": float((Vc * np.abs(F - Fo)).sum() / vol0),
                     "e_shape_rel_diff_vs_oracle": float(
                         abs((Vc * np.abs(F - F0)).sum() - (Vc * np.abs(Fo - F0)).sum())
                         / (Vc * np.abs(Fo - F0)).sum())}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------- other workloads
def _make_trihex(args):
    side, seed, axes, jitter = args
    m = I.trihex_mesh(side, jitter=jitter, seed=seed)
    F = I.init_fraction(m, I.ellipsoid((0.5, 0.5, 0.5), axes), levels=3)
    keep = {k: m[k] for k in ("X", "face_ptr", "face_vert", "owner", "neighbour", "n_cell", "kind")}
    return keep, F


def batch_spec(n_grids=64, seed=20211106):
    """64 distorted triangulated-hex grids of side log-uniform in 16..96,
    interior vertices jittered by U[-0.3h, 0.3h]^3, each with a seeded
    axis-aligned ellipsoid (semi-axes U[0.1, 0.25]) and a uniform velocity
    U[-1, 1]^3."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(16), np.log(96), n_grids))).astype(int)
    axes = rng.uniform(0.1, 0.25, (n_grids, 3))
    vels = rng.uniform(-1.0, 1.0, (n_grids, 3))
    return sides, axes, vels, seed


def batch_inputs(select, procs=16):
    """Meshes and F0 of the selected grids of batch_spec() (generated in a
    spawn process pool, before any CUDA call)."""
    import multiprocessing as mp
    sides, axes, vels, seed = batch_spec()
    jobs = [(int(sides[g]), seed + g, tuple(axes[g]), 0.3) for g in select]
    with mp.get_context("spawn").Pool(max(1, min(procs, os.cpu_count() or 1, len(jobs)))) as pool:
        out = pool.map(_make_trihex, jobs)
    return ([o[0] for o in out], [o[1] for o in out],
            [I.translation(tuple(vels[g])) for g in select], sides[list(select)])


def main_batch(a):
    from paper_2111_01524_gb300 import shard
    ws, rank, local = dist_env()
    all_sides = batch_spec()[0]
    # the grids are independent: each rank takes a share balanced by cells
    parts = shard.balance([float(s) ** 3 for s in all_sides], ws)
    meshes, Fs, vels, sides = batch_inputs(parts[rank])
    import torch
    ws, rank, local, dist = dist_init()
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    n = len(meshes)
    umax = np.array([np.abs(v.u0).max() for v in vels])
    stream = torch.cuda.Stream()
    arms = {}
    for name, prec in (("mixed", V.PREC_MIXED), ("fp64", V.PREC_FP64)):
        ctx = V.Context(meshes, precision=prec)
        cells = int(ctx.n_cell)
        # each grid's step: dt_g = min(CFL 0.5 step, 0.2 / (100 |U|_inf)) so
        # that 100 steps keep every body inside its domain
        with torch.cuda.stream(stream):
            ctx.set_fraction(np.concatenate(Fs))
            ctx.reconstruct()
            t = np.zeros(n)
            dt_cfl = ctx.suggest_dt_batch(vels, t, 0.5, np.full(n, 1e9))
            dt = np.minimum(dt_cfl, 0.2 / (100.0 * umax))
            tuned = ctx.autotune(vels, t, dt, full=True)
            ctx.graph_capture(with_reconstruct=True)
            for _ in range(a.warmup):
                ctx.graph_launch(vels, t, dt)
                t = t + dt
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            clk = ClockSampler(local)
            clk.start()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.steps):
                ctx.graph_launch(vels, t, dt)
                t = t + dt
            e1.record(stream)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            clocks = clk.stop()
            ms = over_ranks(dist, e0.elapsed_time(e1), "max")
            st = ctx.stats()
            F = ctx.get_fraction()
        arms[name] = {"ms": ms, "st": st, "F": F, "clocks": clocks, "faces": int(ctx.n_face),
                      "tuned": {"flux_blocks": tuned[0], "recon_blocks": tuned[1],
                                "faces_per_warp": tuned[2], "prebuilt_polyhedra": tuned[3]}}
        del ctx
        torch.cuda.empty_cache()
    total_cells = over_ranks(dist, cells, "sum")
    dF = over_ranks(dist, float(np.abs(arms["mixed"]["F"] - arms["fp64"]["F"]).max()), "max")
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    mx, f64 = arms["mixed"], arms["fp64"]
    ms, st, clocks = mx["ms"], mx["st"], mx["clocks"]
    v64 = total_cells * a.steps / (f64["ms"] * 1e-3)
    line = {"metric": METRIC, "value": total_cells * a.steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"batch of {len(all_sides)} distorted triangulated-hex grids (side "
                                   "log-uniform 16..96, jitter 0.3h, non-convex cells), ellipsoids, "
                                   "uniform translation, one CUDA graph per step",
                       "cells": int(total_cells), "grids": len(all_sides),
                       "rank0": {"grids": n, "cells": cells, "faces": mx["faces"],
                                 "sides": [int(x) for x in sides]},
                       "parallelism": f"grids sharded over {ws} rank(s) by cells"},
            "autotuned": mx["tuned"],
            "gpu_launches": kernels_per_step(prebuilt=bool(mx["tuned"]["prebuilt_polyhedra"]))
                            * a.steps,
            "band": {"interfacial_cells": st["n_interfacial"], "active_faces": st["n_active_faces"],
                     "truncations_last_step": st["n_truncations"], "overflow": st["n_overflow"],
                     "escaped": st["n_escaped"]},
            "fp64_path": {"value": v64, "unit": UNIT, "ms_per_step": f64["ms"] / a.steps,
                          "mixed_over_fp64": (total_cells * a.steps / (ms * 1e-3)) / v64,
                          "autotuned": f64["tuned"], "clocks": f64["clocks"],
                          "max_abs_F_diff_mixed_vs_fp64": dF,
                          "after_steps": a.warmup + a.steps,
                          "volume_rel_diff_mixed_vs_fp64":
                              (st["volume"] - f64["st"]["volume"]) / f64["st"]["volume"]},
            "clocks": clocks}
    print(json.dumps(line))
    return 0


def main_tets(a):
    """64^3 cubes x 6 jittered Kuhn tets (1.57 M cells), sphere r = 0.15 at
    (0.5, 0.75, 0.5), rigid rotation, CFL 0.4; mixed beside FP64. One
    replica per rank."""
    import torch
    ws, rank, local, dist = dist_init()
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    m = I.kuhn_tet_mesh(64, jitter=0.2, seed=20211105)
    F0 = I.init_fraction(m, I.sphere((0.5, 0.75, 0.5), 0.15), levels=3)
    vel = I.rotation(2 * np.pi)
    res = {}
    for name, prec in (("mixed", V.PREC_MIXED), ("fp64", V.PREC_FP64)):
        ctx = V.Context(m, precision=prec,
                        flux={"emfpa": V.FLUX_EMFPA, "nmfpa": V.FLUX_NMFPA}.get(a.flux, V.FLUX_FMFPA),
                        recon=V.RECON_LSFIR if a.recon == "lsfir" else V.RECON_LSGIR)
        ctx.set_fraction(F0)
        ctx.reconstruct()
        t = 0.0
        for _ in range(a.warmup):
            dt = ctx.suggest_dt(vel, t, 0.4, 1.0)
            ctx.step(vel, t, dt)
            t += dt
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            dt = ctx.suggest_dt(vel, t, 0.4, 1.0)
            ctx.step(vel, t, dt)
            t += dt
        e1.record()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = clk.stop()
        ms = over_ranks(dist, e0.elapsed_time(e1), "max")
        res[name] = {"value": ws * m["n_cell"] * a.steps / (ms * 1e-3), "ms_per_step": ms / a.steps,
                     "F": ctx.get_fraction(), "stats": ctx.stats(), "clocks": clocks}
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": res["mixed"]["value"], "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["mixed"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "64^3 x 6 jittered Kuhn tets, sphere r=0.15 at (0.5,0.75,0.5), "
                                   "rigid rotation, CFL 0.4", "cells": int(m["n_cell"]),
                       "flux_polyhedron": a.flux, "reconstruction": a.recon,
                       "parallelism": f"replicas x{ws}"},
            # tetrahedral grids get no prebuilt candidate lists (many node neighbours)
            "gpu_launches": kernels_per_step(a.recon, prebuilt=False) * a.steps,
            "clocks": res["mixed"]["clocks"],
            "fp64_path": {"value": res["fp64"]["value"],
                          "mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                          "max_abs_F_diff_mixed_vs_fp64":
                              float(np.abs(res["mixed"]["F"] - res["fp64"]["F"]).max())},
            "band": {k: res["mixed"]["stats"][k] for k in ("n_interfacial", "n_active_faces",
                                                           "n_truncations", "n_overflow")}}
    print(json.dumps(line))
    return 0


def main_deform2d(a):
    """2D deformation test (Sec. 4.3) on a quasi-2D grid n x 1 x n (n =
    --grid2d): the cylinder r = 0.15 at (0.5, 0.75) initialised on the device
    (initfgrid, ndiv = 10), the x-z field with period 8, CFL 0.5, steps from
    t = 0; replicas on N GPUs."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    n = a.grid2d
    m = I.slab_mesh(n)
    vel = I.deformation2d(8.0)
    cyl = I.shape_cylinder((0.5, 0.0, 0.75), (0.0, 1.0, 0.0), 0.15)
    res = {}
    for name, prec in (("mixed", V.PREC_MIXED), ("fp64", V.PREC_FP64)):
        ctx = V.Context(m, precision=prec)
        ctx.init_fraction(cyl, 10)  # warm-up of the initialisation
        i0 = torch.cuda.Event(enable_timing=True)
        i1 = torch.cuda.Event(enable_timing=True)
        i0.record()
        ctx.init_fraction(cyl, 10)
        i1.record()
        torch.cuda.synchronize()
        init_ms = i0.elapsed_time(i1)
        ctx.reconstruct()
        t = 0.0
        for _ in range(a.warmup):
            dt = ctx.suggest_dt(vel, t, 0.5, 8.0)
            ctx.step(vel, t, dt)
            t += dt
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        # a small band is launch-bound: the step runs as one CUDA graph (the
        # library's graph of vof_step; dt and t go in through its device
        # table), then as many launched steps for comparison
        stream = torch.cuda.Stream()
        clk = ClockSampler(local)
        clk.start()
        times = {}
        with torch.cuda.stream(stream):
            ctx.graph_capture(with_reconstruct=True)
            for mode in ("graph", "launched"):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(a.steps):
                    dt = ctx.suggest_dt(vel, t, 0.5, 8.0)
                    if mode == "graph":
                        ctx.graph_launch(vel, t, dt)
                    else:
                        ctx.step(vel, t, dt)
                    t += dt
                e1.record(stream)
                stream.synchronize()
                times[mode] = e0.elapsed_time(e1)
                if mode == "graph":
                    F_graph, stats = ctx.get_fraction(), ctx.stats()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = clk.stop()
        ms = over_ranks(dist, times["graph"], "max")
        ms_l = over_ranks(dist, times["launched"], "max")
        res[name] = {"value": ws * m["n_cell"] * a.steps / (ms * 1e-3), "ms_per_step": ms / a.steps,
                     "launched_ms_per_step": ms_l / a.steps,
                     "F": F_graph, "stats": stats, "clocks": clocks, "init_ms": init_ms}
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": res["mixed"]["value"], "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": res["mixed"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"2D deformation (Sec. 4.3), quasi-2D grid {n} x 1 x {n}, "
                                   "cylinder r=0.15 at (0.5, 0.75), period 8, CFL 0.5, steps from t=0",
                       "cells": int(m["n_cell"]), "parallelism": f"replicas x{ws}"},
            "gpu_launches": kernels_per_step() * a.steps, "clocks": res["mixed"]["clocks"],
            "fp64_path": {"value": res["fp64"]["value"],
                          "mixed_over_fp64": res["mixed"]["value"] / res["fp64"]["value"],
                          "max_abs_F_diff_mixed_vs_fp64":
                              float(np.abs(res["mixed"]["F"] - res["fp64"]["F"]).max())},
            "device_init": {"ms": res["mixed"]["init_ms"], "ndiv": 10},
            "step_as": "one CUDA graph per step (vof_graph_capture / vof_graph_launch)",
            "launched": {"ms_per_step": res["mixed"]["launched_ms_per_step"],
                         "fp64_ms_per_step": res["fp64"]["launched_ms_per_step"],
                         "note": "the next steps, each kernel launched from the host"},
            "band": {k: res["mixed"]["stats"][k] for k in ("n_interfacial", "n_active_faces",
                                                           "n_truncations", "n_overflow")}}
    print(json.dumps(line))
    return 0


def _make_request_inputs(args):
    kind, side, seed, body, axes = args
    if kind == "hex":
        m = I.hex_mesh(side)
    else:
        m = I.kuhn_tet_mesh(side, jitter=0.2, seed=seed)
    b = I.sphere((0.5, 0.5, 0.5), 0.15) if body == "sphere" else I.ellipsoid((0.5, 0.5, 0.5), axes)
    F = I.init_fraction(m, b, levels=3)
    keep = {k: m[k] for k in ("X", "face_ptr", "face_vert", "owner", "neighbour", "n_cell", "kind")}
    return keep, F


def serve_trace(n, seed=20211107):
    """The serving request stream: hex or jittered-tet grids (50/50) of
    side log-uniform in 24..160 (tets: side^3 cubes of 6 Kuhn tetrahedra),
    sphere r = 0.15 or an axis-aligned ellipsoid (semi-axes U[0.1, 0.25]),
    field deformation (T = 3) / rotation / translation U[-1, 1]^3, N ~
    U{10..200} steps, CFL 0.5 (0.4 for tets); Poisson arrivals of mean 200
    req/s (first n arrivals)."""
    from paper_2111_01524_gb300 import serve as S
    rng = np.random.default_rng(seed)
    specs = []
    for rid in range(n):
        kind = "hex" if rng.random() < 0.5 else "tet"
        side = int(np.rint(np.exp(rng.uniform(np.log(24), np.log(160)))))
        body = "sphere" if rng.random() < 0.5 else "ellipsoid"
        specs.append((kind, side, seed + rid, body, tuple(rng.uniform(0.1, 0.25, 3))))
    fields = [I.deformation(3.0), I.rotation(2 * np.pi)]

    def make_stub(rid, r):
        which = r.integers(3)
        vel = fields[which] if which < 2 else I.translation(tuple(r.uniform(-1, 1, 3)))
        cfl = 0.4 if specs[rid][0] == "tet" else 0.5
        return S.Request(rid=rid, mesh=None, F0=None, vel=vel, n_steps=int(r.integers(10, 201)),
                         cfl=cfl)

    trace = S.poisson_trace(n, 200.0, seed + 1, make_stub)
    cells = [(s_[1] ** 3) * (6 if s_[0] == "tet" else 1) for s_ in specs]
    return specs, trace, cells


def main_serve(a):
    """The serving workload through the library's device-resident serving
    loop (vof_server_*): the request trace replayed at its arrival times, then
    the same requests with arrivals rescaled to 70% of the capacity the first
    replay measured. Requests are sharded over ranks by estimated cell-steps."""
    import multiprocessing as mp
    from paper_2111_01524_gb300 import serve as S
    from paper_2111_01524_gb300 import shard
    ws, rank, local = dist_env()
    n = a.requests
    specs, trace, cells = serve_trace(n)
    est = [cells[r.rid] * r.n_steps for r in trace]
    mine = shard.balance(est, ws)[rank]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1, len(mine)))) as pool:
        built = pool.map(_make_request_inputs, [specs[i] for i in mine])
    reqs = []
    for i, (m, F) in zip(mine, built):
        r = trace[i]
        r.mesh, r.F0 = m, F
        reqs.append(r)
    import torch
    ws, rank, local, dist = dist_init()
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    free, total = torch.cuda.mem_get_info()
    budget = int(a.budget_frac * free)

    def run(requests, arrivals):
        for r, t in zip(requests, arrivals):
            r.arrival = t
        srv = V.Server(budget_bytes=budget, precision=V.PREC_MIXED, max_batch=a.max_batch)
        if dist is not None:
            dist.barrier()
        clk = ClockSampler(local)
        clk.start()
        st = S.replay(srv, requests)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = clk.stop()
        ss = srv.stats()
        srv.close()
        wall = over_ranks(dist, st.wall, "max")
        cs = over_ranks(dist, st.cell_steps, "sum")
        lat = list(st.latencies)
        if dist is not None:
            allat = [None] * ws
            dist.all_gather_object(allat, lat)
            lat = [x for part in allat for x in part]
        lat = np.asarray(lat) if lat else np.zeros(1)
        return {"value": cs / wall, "wall_s": wall, "cell_steps": cs,
                "p50_ms": float(np.percentile(lat, 50)) * 1e3,
                "p99_ms": float(np.percentile(lat, 99)) * 1e3,
                "ticks": st.ticks, "max_active": ss["max_active"], "batches": ss["n_batches"],
                "batch_steps": ss["batch_steps"],
                # one captured step per live batch per tick (the candidate-list
                # kernel, which batches of tetrahedral grids skip, not counted);
                # a new batch runs its geometry (5), set_fraction (1),
                # reconstruction and velocity setup (1)
                "gpu_launches": int(ss["batch_steps"] * kernels_per_step(prebuilt=False)
                                    + ss["n_batches"] * (5 + 1 + recon_kernels() + 1)),
                "peak_device_bytes": ss["peak_device_bytes"], "budget_bytes": ss["budget_bytes"],
                "budget_bound": bool(ss["peak_device_bytes"] > 0.5 * ss["budget_bytes"]),
                "clocks": clocks}

    arr0 = [r.arrival for r in reqs]
    first = run(reqs, arr0)
    # the same requests at 70% of the measured capacity
    mean_work = float(np.mean([r.n_cell * r.n_steps for r in reqs]))
    rate70 = 0.7 * first["value"] / max(ws, 1) / mean_work
    scale = 200.0 / rate70
    second = run(reqs, [t * scale for t in arr0])
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": first["value"], "unit": UNIT, "n_gpus": ws,
            "steps": int(sum(r.n_steps for r in trace)), "warmup": 0,
            "p50_ms": first["p50_ms"], "p99_ms": first["p99_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"serving: Poisson stream of {n} requests at 200 req/s, hex or "
                                   "jittered-tet grids of side log-uniform 24..160, sphere or "
                                   "ellipsoid, deformation/rotation/translation, N ~ U{10..200} "
                                   f"steps; admitted within {a.budget_frac:.0%} of the free device "
                                   "memory as slots of batched contexts (vof_server_*)",
                       "requests": n, "cells_total": int(sum(cells)),
                       "parallelism": f"requests sharded over {ws} rank(s) by cell-steps"},
            "gpu_launches": first["gpu_launches"],
            "clocks": first["clocks"], "serve": first,
            "serve_70pct": dict(second, rate_req_per_s=rate70)}
    print(json.dumps(line))
    return 0


def cycle_levels(ctx, vel, cfl, t_end):
    """(t, dt) of every step of the run to t_end: Eq. eq:cfl depends on the
    velocity field and t only, so the whole sequence is known up front."""
    out, t = [], 0.0
    while t < t_end - 1e-12:
        dt = ctx.suggest_dt(vel, t, cfl, t_end)
        out.append((t, dt))
        t += dt
    return out


def segment_config(a, counts, n_steps, s0):
    """The workload of the default line (shared by both arms)."""
    return {"workload": f"3D deformation (Enright), uniform hex {a.grid}^3 on the unit cube, "
                        f"sphere r=0.15 at (0.35,0.35,0.35), T=3, CFL 0.5, run to t=3 "
                        f"({n_steps} steps); timed: steps {s0}..{s0 + a.steps - 1}, centred on "
                        f"t=T/2 where the interface sheet is largest",
            "grid": a.grid, "cells": counts["n_cell"], "faces": counts["n_face"],
            "flux_polyhedron": a.flux, "reconstruction": a.recon,
            "parallelism": "replicas x1" if int(os.environ.get("WORLD_SIZE", "1")) == 1
            else f"replicas x{os.environ.get('WORLD_SIZE')}",
            "l2": "inputs larger than L2 (mesh + state ~10 GB), no flush"}


def oracle_state(om, F):
    """The oracle's reconstruction of F (tags, planes) to step from."""
    return om.reconstruct(np.ascontiguousarray(F, np.float64))


def main():
    a = parse()
    if a.impl == "reference":
        return main_reference(a)
    if a.workload == "batch":
        return main_batch(a)
    if a.workload == "tets":
        return main_tets(a)
    if a.workload == "serve":
        return main_serve(a)
    if a.workload == "deform2d":
        return main_deform2d(a)
    if a.workload == "cycle128":
        return main_cycle(a)
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2111_01524_gb300 import build as B
    from paper_2111_01524_gb300 import vof as V
    B.build()
    mesh, F0, vel, cfl, t_end = workload(a.grid)
    counts = I.mesh_counts(mesh)
    prec = V.PREC_MIXED if a.precision == "mixed" else V.PREC_FP64
    flux = {"emfpa": V.FLUX_EMFPA, "nmfpa": V.FLUX_NMFPA}.get(a.flux, V.FLUX_FMFPA)
    recon = V.RECON_LSFIR if a.recon == "lsfir" else V.RECON_LSGIR
    stream = torch.cuda.current_stream()
    F0_dev = torch.from_numpy(F0).cuda()
    K, W = a.steps, a.warmup

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def ctx_from(precision, state=None, F=None):
        c = V.Context(mesh, precision=precision, flux=flux, recon=recon)
        if state is not None:
            c.set_state(state, stream=stream)
        else:
            c.set_fraction(F0_dev if F is None else F, stream=stream)
            c.reconstruct(stream=stream)
        return c

    def timed(ctx, levels, with_phases):
        """W untimed steps, then exactly K steps between two barriers, timed
        with CUDA events on the launching stream."""
        for t, dt in levels[:W]:
            ctx.step(vel, t, dt, stream=stream)
        barrier()
        if with_phases:
            ctx.set_timing(True)
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        per = []
        e0.record(stream)
        for t, dt in levels[W:W + K]:
            s0_ = torch.cuda.Event(enable_timing=True)
            s1_ = torch.cuda.Event(enable_timing=True)
            s0_.record(stream)
            ctx.step(vel, t, dt, stream=stream)
            s1_.record(stream)
            per.append((s0_, s1_))
        e1.record(stream)
        barrier()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1)
        if dist is not None:
            tt = torch.tensor([ms], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        phases = ctx.timing() if with_phases else None
        if with_phases:
            ctx.set_timing(False)
        return ms, [x.elapsed_time(y) for x, y in per], phases, clocks, ctx.stats(stream=stream)

    # ---- A: the whole cycle t = 0 -> 3, one event per step; the state at
    # the start of the timed segment's warm-up is kept (host copies, outside
    # the per-step intervals)
    ctxA = ctx_from(prec)
    levels = cycle_levels(ctxA, vel, cfl, t_end)
    N = len(levels)
    s0 = max(W, N // 2 - K // 2)  # first timed step, centred on t = T/2
    g = ctxA.geometry()
    V_c = g["cell_vol"]
    vol0 = float((V_c * F0).sum())
    band_path = []
    ck = None
    starts, ends = [], []
    ev = torch.cuda.Event(enable_timing=True)
    ev.record(stream)
    for i, (t, dt) in enumerate(levels):
        if i == s0 - W or i % 200 == 0:
            torch.cuda.synchronize()
            st_i = ctxA.stats(stream=stream)
            band_path.append({"step": i, "t": t, "interfacial_cells": st_i["n_interfacial"],
                              "active_faces": st_i["n_active_faces"]})
            if i == s0 - W:
                ck = ctxA.get_state(stream=stream)
                F_ck = ctxA.get_fraction()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        starts.append(ev)
        ctxA.step(vel, t, dt, stream=stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        ends.append(ev)
    torch.cuda.synchronize()
    whole_ms = float(sum(x.elapsed_time(y) for x, y in zip(starts, ends)))
    stA = ctxA.stats(stream=stream)
    FT = ctxA.get_fraction()
    whole = {"steps": N, "ms": whole_ms, "value": ws * counts["n_cell"] * N / (whole_ms * 1e-3),
             "unit": UNIT, "volume_rel_change": (stA["volume"] - vol0) / vol0,
             "clip_loss_rel": stA["clip_loss"] / vol0,
             "e_shape": float((V_c * np.abs(FT - F0)).sum()),
             "band_path": band_path,
             "note": "per-step CUDA-event intervals summed over all steps of the run; host "
                     "read-backs between steps excluded"}
    del ctxA

    # ---- B: the timed segment centred on T/2 (the default line's value)
    seg = levels[s0 - W:s0 + K]
    ctxB = ctx_from(prec, state=ck)
    ms, per_step, phases, clocks, stats = timed(ctxB, seg, True)
    value = ws * counts["n_cell"] * K / (ms * 1e-3)
    FB = ctxB.get_fraction()
    volB = float((V_c * FB).sum())

    # ---- C: the FP64 path on the same segment from the same F (reconstructed
    # by the FP64 path itself: the mixed path's planes would carry its FP32
    # plane constants into the first FP64 step)
    fp64 = None
    if not a.no_fp64 and prec == V.PREC_MIXED:
        c64 = ctx_from(V.PREC_FP64, F=torch.from_numpy(np.ascontiguousarray(F_ck)).cuda())
        ms64, per64, _, clk64, st64 = timed(c64, seg, False)
        v64 = ws * counts["n_cell"] * K / (ms64 * 1e-3)
        F64 = c64.get_fraction()
        fp64 = {"value": v64, "unit": UNIT, "steps": K, "ms_per_step": ms64 / K,
                "mixed_over_fp64": value / v64,
                "band": {"interfacial_cells": st64["n_interfacial"],
                         "active_faces": st64["n_active_faces"]},
                "max_abs_F_diff_mixed_vs_fp64": float(np.abs(FB - F64).max()),
                "l1_rel_F_diff_mixed_vs_fp64": float((V_c * np.abs(FB - F64)).sum()
                                                     / (V_c * F64).sum()),
                "volume_rel_diff_mixed_vs_fp64": float(abs(volB - (V_c * F64).sum()) / vol0),
                "after_steps": W + K,
                "from": f"F at step {s0 - W}, the same for both paths, each reconstructing it"}
        del c64

    # ---- D: the same K steps from t = 0 (the smallest band of the run)
    ctxD = ctx_from(prec)
    msD, _, _, _, stD = timed(ctxD, levels[:W + K], False)
    from_t0 = {"value": ws * counts["n_cell"] * K / (msD * 1e-3), "unit": UNIT,
               "ms_per_step": msD / K, "interfacial_cells": stD["n_interfacial"],
               "active_faces": stD["n_active_faces"]}
    del ctxD

    # ---- E: end to end through the C-ABI with host buffers: each step sets
    # F from pinned host memory, reconstructs, advects, reads F back
    e2e = None
    if not a.no_e2e:
        ctxe = V.Context(mesh, precision=prec, flux=flux, recon=recon)
        Fh = torch.from_numpy(np.ascontiguousarray(F_ck)).pin_memory().numpy()
        ctxe.set_fraction(Fh, stream=stream)
        for t, dt in seg[:W]:
            ctxe.reconstruct(stream=stream)
            ctxe.advect(vel, t, dt, stream=stream)
        ctxe.get_fraction(out=Fh, stream=stream)
        barrier()
        t0 = time.perf_counter()
        for t, dt in seg[W:]:
            ctxe.set_fraction(Fh, stream=stream)
            ctxe.reconstruct(stream=stream)
            ctxe.advect(vel, t, dt, stream=stream)
            ctxe.get_fraction(out=Fh, stream=stream)
        barrier()
        el = time.perf_counter() - t0
        if dist is not None:
            tt = torch.tensor([el], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        e2e = {"value": ws * counts["n_cell"] * K / el, "unit": UNIT,
               "h2d_bytes_per_step": 8 * counts["n_cell"],
               "d2h_bytes_per_step": 8 * counts["n_cell"]}
        del ctxe

    # ---- F: the initial F computed on the device (initfgrid, Sec. 3.2, ndiv = 10)
    init = None
    if not a.no_init:
        ctxi = V.Context(mesh, precision=prec, flux=flux, recon=recon)
        sph = I.shape_sphere((0.35, 0.35, 0.35), 0.15)
        ctxi.init_fraction(sph, 10, stream=stream)  # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctxi.init_fraction(sph, 10, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        Fi = ctxi.get_fraction()
        exact = 4.0 / 3.0 * np.pi * 0.15 ** 3
        init = {"ms": e0.elapsed_time(e1), "ndiv": 10,
                "volume_rel_error": float(abs((V_c * Fi).sum() - exact) / exact),
                "interfacial_cells": int(((Fi > 0) & (Fi < 1)).sum())}
        del ctxi

    # ---- G: the oracle, one step from the state at the segment (CPU baseline;
    # its op counter gives the truncation flops of this step's active faces)
    cpu, oflops = None, None
    if rank == 0 and not a.no_cpu_baseline:
        import oracle
        oracle.build()
        om = oracle.Mesh(mesh)
        st_o = oracle_state(om, F_ck)
        t_ck, dt_ck = seg[0]
        method = {"emfpa": oracle.EMFPA, "nmfpa": oracle.NMFPA}.get(a.flux, oracle.FMFPA)
        rc = oracle.LSFIR if a.recon == "lsfir" else oracle.LSGIR
        t0 = time.perf_counter()
        new = om.step(vel, t_ck, dt_ck, st_o, method=method, recon=rc)
        el = time.perf_counter() - t0
        ostats = new["stats"]
        oflops = {"flops_per_active_face": float(ostats[4]) / max(int(ostats[0]), 1),
                  "flops_per_truncation": float(ostats[4]) / max(int(ostats[3]), 1),
                  "active_faces": int(ostats[0]), "truncations": int(ostats[3])}
        cpu = {"value": om.n_cell / el, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": f"1 full step (faceflux, vofadv, taggrid, LSGIR, plane constants) of "
                         f"the {a.grid}^3 workload from the state at step {s0 - W} (t = "
                         f"{t_ck:.3f}), FP64 C oracle, OpenMP; mesh build and the oracle's "
                         f"reconstruction of that state excluded"}

    peaks, peak_kind = measured_peaks()
    # the dominant kernel: the phase with the longest average launch (the flux
    # phase is its one k_flux launch per step; LSFIR's reconstruction phase
    # takes longer in total but over 1 + 2 n_out shorter launches)
    dom = max(phases.items(), key=lambda kv: kv[1][0] / max(kv[1][1], 1))
    phase = {"name": dom[0], "ms": dom[1][0], "calls": K}
    rl = roofline(stats, phase, counts, peaks, peak_kind, clocks, a.precision, a.flux, oflops)
    launches = sum(n for _, n in phases.values())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": ms / K,
            "p50_ms": float(np.percentile(per_step, 50)),
            "p99_ms": float(np.percentile(per_step, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if a.precision == "mixed" else "f64", "data": "synthetic",
            "config": segment_config(a, counts, N, s0),
            "precision": a.precision,
            "gpu_launches": launches,
            "phases_ms": {k: v[0] for k, v in phases.items()},
            "band": {"interfacial_cells": stats["n_interfacial"],
                     "active_faces": stats["n_active_faces"],
                     "truncations_last_step": stats["n_truncations"],
                     "overflow": stats["n_overflow"], "escaped": stats["n_escaped"],
                     "degenerate_lines_last_step": stats["n_degenerate"],
                     "edge_on_last_step": stats["n_edgeon"],
                     "clipped_last_step": stats["n_clipped"],
                     "reconciled_faces_last_step": stats["n_repaired"]},
            "roofline": rl, "clocks": clocks, "e2e": e2e, "fp64_path": fp64,
            "from_t0": from_t0, "whole_cycle": whole, "device_init": init,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

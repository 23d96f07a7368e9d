"""Host-side arithmetic of bench.py (CPU): the roofline of the dominant kernel
and the kernel count per step that the bench line reports."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


GRID = {"n_cell": 16777216, "n_face": 50528256, "n_vert": 16974593}
COUNTS = {"n_active_faces": 229090, "n_truncations": 355916}
CLOCKS = {"sm_mhz": 2070.0}


def test_flux_roofline_is_truncation_flops_over_one_launch(bench):
    """k_flux runs once per step: 20 steps in 28.47 ms are 1.4235 ms a launch;
    its algorithmic work is 1200 flop per truncation (the construction is the
    polyhedra phase's); the peak is 152 SMs x 128 FP32 lanes x 2 flop x the
    sampled clock."""
    phase = {"name": "flux", "ms": 28.47, "calls": 20}
    r = bench.roofline(COUNTS, phase, GRID, {}, "fallback", CLOCKS, "mixed", "fmfpa")
    fl = 355916 * 1200.0
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["algorithmic_flops_per_launch"] == pytest.approx(fl)
    assert r["achieved"] == pytest.approx(fl / 1.4235e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_flux_roofline_traffic_only_for_the_captured_source(bench, monkeypatch):
    """traffic is the captured bytes per active face times this launch's
    active faces while k_flux.cu is the captured source, and null otherwise."""
    import hashlib
    src = os.path.join(ROOT, "paper_2111_01524_gb300", "csrc", "k_flux.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    phase = {"name": "flux", "ms": 28.47, "calls": 20}
    rec = dict(bench.FLUX_NCU["fmfpa"])
    monkeypatch.setattr(bench, "FLUX_NCU", {"fmfpa": dict(rec, source_sha256=sha)})
    r = bench.roofline(COUNTS, phase, GRID, {}, "fallback", CLOCKS, "mixed", "fmfpa")
    assert r["traffic"] == pytest.approx(rec["dram_bytes_per_active_face"] * 229090)
    assert r["ncu"]["capture"].startswith("profiles/")
    assert os.path.exists(os.path.join(ROOT, r["ncu"]["capture"]))
    monkeypatch.setattr(bench, "FLUX_NCU", {"fmfpa": dict(rec, source_sha256="0" * 64)})
    r = bench.roofline(COUNTS, phase, GRID, {}, "fallback", CLOCKS, "mixed", "fmfpa")
    assert r["traffic"] is None and r["ncu"] is None
    # every record names a committed capture
    for kind, rec in bench.FLUX_NCU.items():
        assert os.path.exists(os.path.join(ROOT, rec["capture"])), kind


def test_sweep_roofline_is_hbm_bytes_over_one_launch(bench):
    """A sweep phase is reported against the measured copy bandwidth with its
    algorithmic bytes (cell tags: read F, write the tag, 9 B per cell)."""
    phase = {"name": "cell_tags", "ms": 2.0, "calls": 10}
    r = bench.roofline(COUNTS, phase, GRID, {"hbm_gbs": 6684.8}, "measured", CLOCKS, "mixed")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(GRID["n_cell"] * 9 / 0.2e-3 / 1e9)
    assert r["peak"] == 6684.8


def test_kernels_per_step(bench):
    """LSGIR: cell tags 1, node tags 3, reconstruct 1, face sweep 2,
    polyhedra 1, flux 1, update 2 = 11; LSFIR replaces the reconstruction's
    1 by 1 + 2 per outer iteration; the mixed path adds the closed form of
    the box cells' plane constants (1), the reconciliation of FP32 noise (16:
    3 rounds of 5 and the final clip) and, with prebuilt polyhedra, their
    candidate lists (1)."""
    assert bench.kernels_per_step(precision="fp64") == 11
    assert bench.kernels_per_step("lsfir", 4, precision="fp64") == 19
    assert bench.kernels_per_step("lsfir", 1, precision="fp64") == 13
    assert bench.kernels_per_step() == 11 + 1 + 16 + 1
    assert bench.kernels_per_step(prebuilt=False) == 11 + 1 + 16
    assert bench.kernels_per_step("lsfir", 4) == 19 + 16 + 1
    assert bench.recon_kernels(precision="fp64") + bench.advect_kernels("fp64") == 11


def test_flux_roofline_uses_the_oracle_op_count(bench):
    """With the oracle's op count of the same state's truncations, the
    numerator is its flops per active face times the launch's active faces."""
    counts = dict(COUNTS)
    phase = {"name": "flux", "ms": 10.0, "calls": 10}
    ofl = {"flops_per_active_face": 27000.0, "flops_per_truncation": 13000.0}
    r = bench.roofline(counts, phase, GRID, {"hbm_gbs": 6684.8}, "measured", CLOCKS, "mixed",
                       "fmfpa", ofl)
    assert r["algorithmic_flops_per_launch"] == counts["n_active_faces"] * 27000.0
    assert "oracle op counter" in r["flops_source"]
    assert r["achieved"] == pytest.approx(counts["n_active_faces"] * 27000.0 / 1e-3 / 1e12)

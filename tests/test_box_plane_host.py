"""The closed-form plane constant of an axis-aligned box (the mixed path's
box cells), run on the host against the oracle.

The FP32 functions of csrc/box_plane.cuh are host-callable; a small driver
(tests/host/box_plane_host.cu, built with nvcc for the host only) solves
V(g) = v for slopes m of the unit cube, and the oracle's FP64 clip of a unit
cube cell by the plane {m.u <= g} must give v back (Eq. plic-eq). The cases
cover the regimes of the volume function: a corner (tiny v), slopes of zero
(a plane parallel to one or two axes), a tiny smallest slope (the cancellation
the piecewise integration avoids), equal slopes, the centre (v = 1/2), and
random slopes, with v from 1e-12 up.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2111_01524_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))

# relative to v: the FP32 root and volume function, a few 1e-7; absolute
# (of the unit cell): the oracle's clip and a plane across a whole face
REL = 1e-5
ABS = 1e-13


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("boxh") / "box_plane_host")
    r = subprocess.run([nvcc, "-O2", "-x", "cu", os.path.join(HERE, "host", "box_plane_host.cu"),
                        "-o", exe], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    return exe


def _cases(seed=7):
    rng = np.random.default_rng(seed)
    ms = [(0.0, 0.0, 1.0), (0.0, 0.3, 0.7), (1e-9, 0.25, 0.75), (1e-6, 1e-6, 1.0),
          (1e-3, 0.4, 0.6), (1 / 3, 1 / 3, 1 / 3), (0.2, 0.3, 0.5), (0.05, 0.05, 0.9)]
    for _ in range(40):
        w = rng.dirichlet((1.0, 1.0, 1.0))
        if rng.random() < 0.3:
            w[0] *= 10.0 ** rng.uniform(-9, -2)
        ms.append(tuple(w / w.sum()))
    vs = [0.0, 1e-12, 1e-9, 1e-6, 1e-3, 0.02, 0.1, 0.25, 0.4, 0.49, 0.5]
    out = []
    for m in ms:
        m1, m2 = np.float32(m[0]), np.float32(m[1])
        m3 = np.float32(1.0 - float(m1) - float(m2))
        for v in vs + list(10.0 ** rng.uniform(-12, np.log10(0.5), 3)):
            out.append((m1, m2, m3, np.float32(v)))
    return out


def test_box_root_cuts_the_fraction(driver, orc):
    cases = _cases()
    text = "".join(f"{a:.9g} {b:.9g} {c:.9g} {v:.9g}\n" for a, b, c, v in cases)
    r = subprocess.run([driver], input=text, capture_output=True, text=True, check=True)
    rows = np.array([list(map(float, ln.split())) for ln in r.stdout.splitlines()])
    assert rows.shape == (len(cases), 5)
    om = orc.Mesh(I.hex_mesh(1))  # the unit cube, centroid (1/2, 1/2, 1/2)
    for (m1, m2, m3, v), (b1, b2, b3, g, it) in zip(cases, rows):
        want = [x if x >= np.float32(1e-20) else np.float32(0) for x in sorted([m1, m2, m3])]
        got = [np.float32(b) for b in (b1, b2, b3)]  # 9 digits print a float exactly
        assert got == want
        m = np.array(got, np.float64)
        nm = np.linalg.norm(m)
        # {m.u <= g} is {n.(u - x_c) + C >= 0} with n = -m/|m|, C = (g - m.x_c)/|m|
        V = om.cell_cut_volume(0, -m / nm, (g - 0.5 * m.sum()) / nm)
        assert abs(V - float(v)) <= REL * float(v) + ABS, (m1, m2, m3, v, g, V)
        assert 0.0 <= g <= 0.5
        assert it <= 3  # at most four evaluations of V from the closed-form bracket


def test_box_root_degenerate_ends(driver):
    """v = 0 gives the corner itself, v = 1/2 the centre plane."""
    text = "0.2 0.3 0.5 0\n0.2 0.3 0.5 0.5\n0 0 1 0.5\n0 0 1 0\n"
    r = subprocess.run([driver], input=text, capture_output=True, text=True, check=True)
    g = [float(ln.split()[3]) for ln in r.stdout.splitlines()]
    assert g[0] == 0.0 and g[3] == 0.0
    assert g[1] == pytest.approx(0.5, abs=1e-7) and g[2] == pytest.approx(0.5, abs=1e-7)

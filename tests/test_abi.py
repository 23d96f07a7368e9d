"""CPU checks of the C-ABI library: it builds, loads, and exports every
symbol that include/vof.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vof_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    from paper_2111_01524_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "vof_init" in syms and "vof_advect" in syms and "vof_reconstruct" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_the_boundary_calls_are_exported():
    """The calls of the C-ABI boundary: context, state, the method's steps,
    batching, serving and the read-backs."""
    from paper_2111_01524_gb300 import build
    lib = ctypes.CDLL(build.build())
    for s in ("vof_init", "vof_destroy", "vof_last_error", "vof_set_fraction", "vof_get_fraction",
              "vof_reconstruct", "vof_advect_step", "vof_suggest_dt", "vof_get_planes",
              "vof_get_face_flux", "vof_get_candidates", "vof_get_state", "vof_set_state",
              "vof_batch_create", "vof_batch_step", "vof_server_create", "vof_server_submit",
              "vof_server_step", "vof_server_poll", "vof_server_get_stats", "vof_server_destroy",
              "vof_estimate_bytes", "vof_get_stats"):
        assert hasattr(lib, s), s
    assert "vof_init" in declared_symbols() and "vof_server_submit" in declared_symbols()


def test_server_options_are_checked_on_the_host():
    from paper_2111_01524_gb300 import vof
    for kw in ({"precision": 5}, {"budget_bytes": -1}, {"max_batch": -2}):
        with pytest.raises(vof.VofError) as e:
            vof.Server(**kw)
        assert e.value.status == vof.VOF_EINVAL


def test_server_checks_a_request_mesh_on_submit():
    """The structure of a request's mesh is checked on the host when it is
    submitted (its connectivity is built later, once, at admission)."""
    import numpy as np
    from paper_2111_01524_gb300 import inputs as I, vof
    srv = vof.Server(budget_bytes=1 << 30)
    try:
        m = I.hex_mesh(3)
        F0 = np.zeros(27)
        assert srv.submit(m, F0, I.rotation(1.0), 5) == 0
        bad = dict(m, owner=np.array(m["owner"]).copy())
        bad["owner"][4] = 27  # not a cell
        with pytest.raises(vof.VofError) as e:
            srv.submit(bad, F0, I.rotation(1.0), 5)
        assert e.value.status == vof.VOF_EINVAL
        bad = dict(m, face_vert=np.array(m["face_vert"]).copy())
        bad["face_vert"][0] = -1
        with pytest.raises(vof.VofError):
            srv.submit(bad, F0, I.rotation(1.0), 5)
        assert srv.stats()["n_submitted"] == 1
    finally:
        srv.close()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2111_01524_gb300 import build, vof
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(vof, "_lib", None)
    try:
        vof.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:  # pragma: no cover
        raise AssertionError("expected a loud failure")


def test_status_codes_match_header():
    from paper_2111_01524_gb300 import vof
    src = open(os.path.join(ROOT, "include", "vof.h")).read()
    for name, val in [("VOF_OK", vof.VOF_OK), ("VOF_EINVAL", vof.VOF_EINVAL),
                      ("VOF_ENOMEM", vof.VOF_ENOMEM), ("VOF_ECUDA", vof.VOF_ECUDA),
                      ("VOF_ECAPACITY", vof.VOF_ECAPACITY), ("VOF_ESTATE", vof.VOF_ESTATE),
                      ("VOF_ECFL", vof.VOF_ECFL)]:
        assert re.search(rf"{name}\s*=\s*{val}\b", src), name


def test_struct_layouts():
    from paper_2111_01524_gb300 import vof
    assert ctypes.sizeof(vof._Mesh) == 3 * 8 + 5 * 8
    assert ctypes.sizeof(vof._Opt) == 8 + 8 + 4 + 4 + 4 + 4 + 8 + 2 * 4
    assert ctypes.sizeof(vof._Vel) == 4 + 4 + 8 + 8 + 24 + 24
    assert ctypes.sizeof(vof.Stats) == 6 * 8 + 5 * 8 + 3 * 8
    assert ctypes.sizeof(vof._Shape) == 4 + 4 + 24 + 24 + 8


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and field offsets of the binding's structs equal the C header's
    (compiled here with the host compiler)."""
    import shutil
    import subprocess
    from paper_2111_01524_gb300 import vof
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"vof_mesh_desc": vof._Mesh, "vof_options": vof._Opt, "vof_velocity": vof._Vel,
               "vof_stats": vof.Stats, "vof_shape": vof._Shape}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vof.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_flux_constants_match_header():
    from paper_2111_01524_gb300 import vof
    src = open(os.path.join(ROOT, "include", "vof.h")).read()
    assert re.search(rf"VOF_FLUX_FMFPA\s*=\s*{vof.FLUX_FMFPA}\b", src)
    assert re.search(rf"VOF_FLUX_EMFPA\s*=\s*{vof.FLUX_EMFPA}\b", src)
    assert re.search(rf"VOF_FLUX_NMFPA\s*=\s*{vof.FLUX_NMFPA}\b", src)
    assert re.search(rf"VOF_MAX_POLY_VERTS\s*=\s*{vof.NB_VERTS}\b", src)
    assert re.search(rf"VOF_RECON_LSGIR\s*=\s*{vof.RECON_LSGIR}\b", src)
    assert re.search(rf"VOF_RECON_LSFIR\s*=\s*{vof.RECON_LSFIR}\b", src)
    from paper_2111_01524_gb300 import inputs as I
    for name, val in (("SPHERE", I.Shape.SPHERE), ("CYLINDER", I.Shape.CYLINDER),
                      ("HALFSPACE", I.Shape.HALFSPACE)):
        assert re.search(rf"VOF_SHAPE_{name}\s*=\s*{val}\b", src), name
    # 3I+1 EMFPA points for I <= 6, 2I+1 FMFPA points for I <= 8
    assert vof.NB_VERTS >= max(3 * 6 + 1, 2 * 8 + 1)


def test_timing_phases_match_header():
    """vof.Context.timing() names the phases in the order of VOF_PHASE_*,
    and asks for all VOF_NUM_PHASES of them."""
    from paper_2111_01524_gb300 import vof
    src = open(os.path.join(ROOT, "include", "vof.h")).read()
    found = {m.group(1).lower(): int(m.group(2))
             for m in re.finditer(r"VOF_PHASE_([A-Z_]+)\s*=\s*(\d+)", src)}
    n = int(re.search(r"VOF_NUM_PHASES\s*=\s*(\d+)", src).group(1))
    assert len(vof.Context.PHASES) == n == len(found)
    for i, name in enumerate(vof.Context.PHASES):
        assert found[name] == i, name


def _heptagonal_prism():
    """one cell: two 7-node faces and seven quads (valid orientation)"""
    import numpy as np
    a = 2 * np.pi * np.arange(7) / 7
    ring = np.stack([0.5 + 0.4 * np.cos(a), 0.5 + 0.4 * np.sin(a)], 1)
    X = np.concatenate([np.c_[ring, np.zeros(7)], np.c_[ring, np.ones(7)]])
    loops = [list(range(6, -1, -1)), list(range(7, 14))]
    loops += [[i, (i + 1) % 7, 7 + (i + 1) % 7, 7 + i] for i in range(7)]
    fp = np.cumsum([0] + [len(l) for l in loops]).astype(np.int64)
    return {"X": X, "face_ptr": fp, "face_vert": np.concatenate(loops).astype(np.int32),
            "owner": np.zeros(len(loops), np.int32),
            "neighbour": np.full(len(loops), -1, np.int32), "n_cell": 1}


def test_emfpa_and_bad_options_are_rejected_before_device_work():
    """vof_init checks the options before it touches the device: EMFPA on a
    mesh with a 7-node face, an unknown construction or reconstruction and
    LSFIR limits out of range each give VOF_EINVAL (no GPU needed)."""
    from paper_2111_01524_gb300 import vof
    m = _heptagonal_prism()
    with pytest.raises(vof.VofError) as e:
        vof.Context(m, flux=vof.FLUX_EMFPA)
    assert e.value.status == vof.VOF_EINVAL and "6 nodes" in str(e.value)
    with pytest.raises(vof.VofError) as e:
        vof.Context(m, flux=7)
    assert e.value.status == vof.VOF_EINVAL
    for bad in ({"recon": 2}, {"recon": vof.RECON_LSFIR, "lsfir_max_iter": 17},
                {"recon": vof.RECON_LSFIR, "lsfir_max_iter": -1},
                {"recon": vof.RECON_LSFIR, "lsfir_tol": -1e-3}):
        with pytest.raises(vof.VofError) as e:
            vof.Context(m, **bad)
        assert e.value.status == vof.VOF_EINVAL, bad


def test_corrupted_meshes_are_rejected_before_device_work():
    """vof_init validates the face-based mesh on the host before it touches
    the device: a CSR that does not start at 0, faces of fewer than 3 or
    more than 8 nodes (a non-monotone CSR shows up as one of these), an
    owner out of range, a face whose neighbour is its owner, a node index
    out of range and an empty mesh each give VOF_EINVAL with a message (no
    GPU needed)."""
    import numpy as np
    from paper_2111_01524_gb300 import inputs as I
    from paper_2111_01524_gb300 import vof
    base = I.hex_mesh(2)

    def bad(**kw):
        m = {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in base.items()}
        for k, f in kw.items():
            f(m)
        with pytest.raises(vof.VofError) as e:
            vof.Context(m)
        assert e.value.status == vof.VOF_EINVAL
        assert str(e.value)
        return str(e.value)

    def shift_ptr(m):
        m["face_ptr"] = m["face_ptr"] + 1
    assert "face_ptr[0]" in bad(a=shift_ptr)

    def two_nodes(m):
        fp = m["face_ptr"].copy()
        fp[1] = fp[0] + 2  # face 0 keeps 2 nodes, face 1 gets 6
        m["face_ptr"] = fp
    assert "nodes" in bad(a=two_nodes)

    def non_monotone(m):
        fp = m["face_ptr"].copy()
        fp[2], fp[3] = fp[3], fp[2]
        m["face_ptr"] = fp
    assert "nodes" in bad(a=non_monotone)

    def owner_out(m):
        m["owner"][0] = m["n_cell"]
    assert "owner" in bad(a=owner_out)

    def self_neighbour(m):
        f = int(np.nonzero(m["neighbour"] >= 0)[0][0])
        m["neighbour"][f] = m["owner"][f]
    assert "owner" in bad(a=self_neighbour)

    def node_out(m):
        m["face_vert"][5] = len(m["X"])
    assert "out of range" in bad(a=node_out)

    def empty(m):
        m["n_cell"] = 0
    bad(a=empty)

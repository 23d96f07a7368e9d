"""Oracle for the unsplit geometric VOF step -- TEST INFRASTRUCTURE ONLY.

Python binding (ctypes) of the plain FP64 C oracle in ``oracle.c``. Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package; the product path never does. It shares no code with
the CUDA library: both sides only read the seeded inputs of
``paper_2111_01524_gb300.inputs``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

# flux polyhedron constructions of faceflux / step
FMFPA = 0  # face-matched (Sec. 2.2.2)
EMFPA = 1  # edge-matched (Sec. 2.2.1)
NMFPA = 2  # non-matched (Sec. 2.2.3)
# interface reconstructions of reconstruct / step
LSGIR = 0  # least-squares gradient (Sec. 2.1.1)
LSFIR = 1  # least-squares fit with the outer iteration (Sec. 2.1.2)
_lib = None


def build(force=False):
    """Compile the oracle with gcc (plain IEEE FP64: no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Vel(C.Structure):
    _fields_ = [("kind", C.c_int), ("pad", C.c_int), ("period", C.c_double),
                ("omega", C.c_double), ("center", C.c_double * 3), ("u0", C.c_double * 3)]


def _vel(v):
    s = _Vel()
    s.kind = v.kind
    s.period = v.period
    s.omega = v.omega
    for i in range(3):
        s.center[i] = v.center[i]
        s.u0[i] = v.u0[i]
    return s


class _Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("pad", C.c_int), ("c", C.c_double * 3),
                ("a", C.c_double * 3), ("r", C.c_double)]


def _body(b):
    s = _Body()
    s.kind = b.kind
    for i in range(3):
        s.c[i] = b.c[i]
        s.a[i] = b.a[i]
    s.r = b.r
    return s


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
        L.orc_mesh_build.restype = vp
        L.orc_mesh_build.argtypes = [i64, vp, i64, vp, vp, vp, vp, i64]
        L.orc_mesh_free.argtypes = [vp]
        L.orc_geometry.argtypes = [vp] + [vp] * 7
        L.orc_neighbors.restype = i64
        L.orc_neighbors.argtypes = [vp, vp, vp]
        L.orc_candidates.restype = i32
        L.orc_candidates.argtypes = [vp, i64, vp, i32]
        L.orc_taggrid.argtypes = [vp, dbl, vp, vp, vp, vp, vp]
        L.orc_lsgir.argtypes = [vp, dbl, vp, vp, vp]
        L.orc_plane_constant.argtypes = [vp, vp, vp, vp, vp]
        L.orc_cell_cut_volume.restype = dbl
        L.orc_cell_cut_volume.argtypes = [vp, i64, vp, dbl]
        L.orc_velocity_eval.argtypes = [vp, vp, dbl, vp]
        L.orc_fmfpa.restype = i32
        L.orc_fmfpa.argtypes = [vp, i64, vp, dbl, dbl, vp, i32, vp, vp]
        L.orc_initfgrid.argtypes = [vp, vp, i32, vp]
        L.orc_plic_centre.restype = i32
        L.orc_plic_centre.argtypes = [vp, i64, vp, dbl, vp]
        L.orc_lsfir_normals.restype = i64
        L.orc_lsfir_normals.argtypes = [vp, vp, vp, vp, vp]
        L.orc_lsfir_accept.restype = dbl
        L.orc_lsfir_accept.argtypes = [vp, vp, i32, vp, vp]
        L.orc_lsfir.restype = i32
        L.orc_lsfir.argtypes = [vp, i32, dbl, vp, vp, vp, vp]
        L.orc_nmfpa.restype = i32
        L.orc_nmfpa.argtypes = [vp, i64, vp, dbl, dbl, vp, i32, vp, vp]
        L.orc_emfpa.restype = i32
        L.orc_emfpa.argtypes = [vp, i64, vp, dbl, dbl, vp, i32, vp, vp]
        L.orc_faceflux.argtypes = [vp, vp, dbl, dbl, vp, vp, vp, vp, vp, vp, vp, vp, i32]
        L.orc_vofadv.argtypes = [vp, vp, vp, vp]
        L.orc_suggest_dt.restype = dbl
        L.orc_suggest_dt.argtypes = [vp, vp, dbl, dbl, dbl]
        L.orc_poly_clip_volume.restype = dbl
        L.orc_poly_clip_volume.argtypes = [i32, vp, i32, vp, vp, i32, vp]
        L.orc_poly_volume.restype = dbl
        L.orc_poly_volume.argtypes = [i32, vp, i32, vp, vp]
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def num_threads():
    return lib().orc_num_threads()


class Mesh:
    """Oracle view of a face-based mesh (Sec. 3.1): connectivity + geometry."""

    def __init__(self, mesh):
        L = lib()
        self._keep = dict(
            X=np.ascontiguousarray(mesh["X"], np.float64),
            fp=np.ascontiguousarray(mesh["face_ptr"], np.int64),
            fv=np.ascontiguousarray(mesh["face_vert"], np.int32),
            own=np.ascontiguousarray(mesh["owner"], np.int32),
            nbr=np.ascontiguousarray(mesh["neighbour"], np.int32),
        )
        k = self._keep
        self.n_vert = k["X"].shape[0]
        self.n_face = k["own"].shape[0]
        self.n_cell = int(mesh["n_cell"])
        self.h = None
        self._m = L.orc_mesh_build(self.n_vert, _p(k["X"]), self.n_face, _p(k["fp"]),
                                   _p(k["fv"]), _p(k["own"]), _p(k["nbr"]), self.n_cell)
        if not self._m:
            raise ValueError("oracle: invalid mesh")
        self._geo = None

    def __del__(self):
        if getattr(self, "_m", None):
            lib().orc_mesh_free(self._m)
            self._m = None

    def geometry(self):
        if self._geo is None:
            nc, nf = self.n_cell, self.n_face
            g = dict(cell_vol=np.empty(nc), cell_cen=np.empty((nc, 3)),
                     face_cen=np.empty((nf, 3)), face_nrm=np.empty((nf, 3)),
                     face_area=np.empty(nf), cell_bbox=np.empty((nc, 6)),
                     cell_convex=np.empty(nc, np.uint8))
            lib().orc_geometry(self._m, _p(g["cell_vol"]), _p(g["cell_cen"]), _p(g["face_cen"]),
                               _p(g["face_nrm"]), _p(g["face_area"]), _p(g["cell_bbox"]),
                               _p(g["cell_convex"]))
            self._geo = g
        return self._geo

    def neighbors(self):
        L = lib()
        n = L.orc_neighbors(self._m, None, None)
        ptr = np.empty(self.n_cell + 1, np.int64)
        idx = np.empty(max(n, 1), np.int32)
        L.orc_neighbors(self._m, _p(ptr), _p(idx))
        return ptr, idx[:n]

    def candidates(self, face):
        buf = np.empty(8192, np.int32)
        n = lib().orc_candidates(self._m, int(face), _p(buf), 8192)
        return buf[:min(n, 8192)].copy()

    # --- taggrid / reconstruction (Secs. 3.3, 2.1, 2.1.1)
    def taggrid(self, F, eps=1e-12):
        F = np.array(F, np.float64, copy=True)
        Fn = np.empty(self.n_vert)
        tv = np.empty(self.n_vert, np.int8)
        tf = np.empty(self.n_face, np.int8)
        tc = np.empty(self.n_cell, np.int8)
        lib().orc_taggrid(self._m, eps, _p(F), _p(Fn), _p(tv), _p(tf), _p(tc))
        return dict(F=F, Fnode=Fn, tag_v=tv, tag_f=tf, tag_c=tc)

    def lsgir(self, F, tag_c, beta=1.5):
        F = np.ascontiguousarray(F, np.float64)
        tag_c = np.ascontiguousarray(tag_c, np.int8)
        n = np.empty((self.n_cell, 3))
        lib().orc_lsgir(self._m, beta, _p(F), _p(tag_c), _p(n))
        return n

    def plane_constant(self, F, tag_c, nrm):
        F = np.ascontiguousarray(F, np.float64)
        tag_c = np.ascontiguousarray(tag_c, np.int8)
        nrm = np.ascontiguousarray(nrm, np.float64)
        Cc = np.empty(self.n_cell)
        lib().orc_plane_constant(self._m, _p(F), _p(tag_c), _p(nrm), _p(Cc))
        return Cc

    def cell_cut_volume(self, cell, n, Cval):
        n = np.ascontiguousarray(n, np.float64)
        return lib().orc_cell_cut_volume(self._m, int(cell), _p(n), float(Cval))

    def initfgrid(self, shape, ndiv=10):
        """initial F by refinement (Sec. 3.2): ndiv^3 pieces per tetrahedron of
        each cell near the surface of ``shape`` (inputs.Shape)."""
        F = np.empty(self.n_cell)
        b = _body(shape)
        lib().orc_initfgrid(self._m, C.byref(b), int(ndiv), _p(F))
        return F

    def plic_centre(self, cell, n, Cval):
        """vertex average of the PLIC polygon of a cell (Sec. 2.1.2)"""
        out = np.empty(3)
        n = np.ascontiguousarray(n, np.float64)  # held while C reads it
        k = lib().orc_plic_centre(self._m, int(cell), _p(n), float(Cval), _p(out))
        return out, int(k)

    def lsfir_normals(self, tag_c, nrm, xp):
        """one LSFIR normal update from the PLIC centres xp (Sec. 2.1.2)"""
        cand = np.empty((self.n_cell, 3))
        tag_c = np.ascontiguousarray(tag_c, np.int8)
        nrm = np.ascontiguousarray(nrm, np.float64)
        xp = np.ascontiguousarray(xp, np.float64)
        kept = lib().orc_lsfir_normals(self._m, _p(tag_c), _p(nrm), _p(xp), _p(cand))
        return cand, int(kept)

    def lsfir_accept(self, tag_c, io, cand, nrm):
        """acceptance step of outer iteration io (Sec. 2.1.2); returns the
        new normals and the largest accepted turn"""
        out = np.array(nrm, np.float64, copy=True)
        tag_c = np.ascontiguousarray(tag_c, np.int8)
        cand = np.ascontiguousarray(cand, np.float64)
        t = lib().orc_lsfir_accept(self._m, _p(tag_c), int(io), _p(cand), _p(out))
        return out, float(t)

    def lsfir(self, F, tag_c, nrm0, n_out=4, tol=1e-3):
        """LSFIR outer iteration from the normals nrm0 (Sec. 2.1.2)."""
        nrm = np.array(nrm0, np.float64, copy=True)
        Cc = np.empty(self.n_cell)
        F = np.ascontiguousarray(F, np.float64)
        tag_c = np.ascontiguousarray(tag_c, np.int8)
        it = lib().orc_lsfir(self._m, int(n_out), float(tol), _p(F), _p(tag_c), _p(nrm), _p(Cc))
        return nrm, Cc, int(it)

    def reconstruct(self, F, eps=1e-12, beta=1.5, recon=LSGIR, n_out=4, tol=1e-3):
        """taggrid + lsgir + volume enforcement: the reconstruction half-step;
        recon = LSFIR adds the least-squares fit outer iteration (Sec. 2.1.2,
        n_out repetitions at most, tolerance tol in radians)."""
        st = self.taggrid(F, eps)
        st["nrm"] = self.lsgir(st["F"], st["tag_c"], beta)
        if recon == LSFIR:
            st["nrm"], st["C"], st["lsfir_iters"] = self.lsfir(st["F"], st["tag_c"], st["nrm"],
                                                               n_out, tol)
        else:
            st["C"] = self.plane_constant(st["F"], st["tag_c"], st["nrm"])
        return st

    # --- advection (Secs. 2.2, 3.5)
    def fmfpa(self, face, vel, t_half, dt):
        out = np.empty((65, 3))
        vd = np.zeros(1)
        fl = np.zeros(1, np.int32)
        v = _vel(vel)
        I = lib().orc_fmfpa(self._m, int(face), C.byref(v), t_half, dt, _p(out), 32, _p(vd), _p(fl))
        if I < 0:
            raise ValueError("face too large")
        return out[:2 * I + 1].copy(), float(vd[0]), int(fl[0])

    def emfpa(self, face, vel, t_half, dt):
        """EMFPA flux polyhedron (Sec. 2.2.1): 3I+1 points."""
        out = np.empty((97, 3))
        vd = np.zeros(1)
        fl = np.zeros(1, np.int32)
        v = _vel(vel)
        I = lib().orc_emfpa(self._m, int(face), C.byref(v), t_half, dt, _p(out), 32, _p(vd), _p(fl))
        if I < 0:
            raise ValueError("face too large")
        return out[:3 * I + 1].copy(), float(vd[0]), int(fl[0])

    def nmfpa(self, face, vel, t_half, dt):
        """NMFPA flux polyhedron (Sec. 2.2.3): 2I points."""
        out = np.empty((64, 3))
        vd = np.zeros(1)
        fl = np.zeros(1, np.int32)
        v = _vel(vel)
        I = lib().orc_nmfpa(self._m, int(face), C.byref(v), t_half, dt, _p(out), 32, _p(vd), _p(fl))
        if I < 0:
            raise ValueError("face too large")
        return out[:2 * I].copy(), float(vd[0]), int(fl[0])

    def faceflux(self, vel, t, dt, st, method=FMFPA):
        Vd = np.empty(self.n_face)
        VF = np.empty(self.n_face)
        stats = np.zeros(5, np.int64)
        v = _vel(vel)
        lib().orc_faceflux(self._m, C.byref(v), t, dt, _p(st["F"]), _p(st["tag_f"]),
                           _p(st["tag_c"]), _p(st["nrm"]), _p(st["C"]), _p(Vd), _p(VF),
                           _p(stats), int(method))
        return Vd, VF, stats

    def vofadv(self, F, Vd, VF):
        F = np.array(F, np.float64, copy=True)
        lib().orc_vofadv(self._m, _p(np.ascontiguousarray(Vd)), _p(np.ascontiguousarray(VF)), _p(F))
        return F

    def suggest_dt(self, vel, t, cfl, t_end):
        v = _vel(vel)
        return lib().orc_suggest_dt(self._m, C.byref(v), t, cfl, t_end)

    def velocity(self, vel, x, t):
        v = _vel(vel)
        x = np.ascontiguousarray(x, np.float64)
        u = np.empty(3)
        lib().orc_velocity_eval(C.byref(v), _p(x), t, _p(u))
        return u

    def step(self, vel, t, dt, st, eps=1e-12, beta=1.5, method=FMFPA, recon=LSGIR):
        """One time step of the advection test loop (Algorithm alg:adv):
        faceflux -> vofadv -> taggrid -> lsgir [-> lsfir] -> volume enforcement.
        method: the flux polyhedron, FMFPA (Sec. 2.2.2), EMFPA (Sec. 2.2.1) or
        NMFPA (Sec. 2.2.3);
        recon: LSGIR (Sec. 2.1.1) or LSFIR (Sec. 2.1.2)."""
        Vd, VF, stats = self.faceflux(vel, t, dt, st, method)
        F = self.vofadv(st["F"], Vd, VF)
        new = self.reconstruct(F, eps, beta, recon)
        new["Vd"], new["VF"], new["stats"] = Vd, VF, stats
        new["F_unclipped_cut"] = F
        return new


def poly_volume(verts, faces):
    verts = np.ascontiguousarray(verts, np.float64)
    fp = np.cumsum([0] + [len(f) for f in faces]).astype(np.int32)
    fi = np.ascontiguousarray(np.concatenate(faces), np.int32)
    return lib().orc_poly_volume(len(verts), _p(verts), len(faces), _p(fp), _p(fi))


def poly_clip_volume(verts, faces, planes):
    """Volume of P ∩ {a.x + b > 0 for each plane (a, b)} (winding number)."""
    verts = np.ascontiguousarray(verts, np.float64)
    fp = np.cumsum([0] + [len(f) for f in faces]).astype(np.int32)
    fi = np.ascontiguousarray(np.concatenate(faces), np.int32)
    pl = np.ascontiguousarray(np.asarray(planes, np.float64).reshape(-1, 4))
    return lib().orc_poly_clip_volume(len(verts), _p(verts), len(faces), _p(fp), _p(fi),
                                      pl.shape[0], _p(pl))

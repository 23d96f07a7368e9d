"""Thin ctypes binding of the gvof CUDA library (``include/vof.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels. Device buffers are torch tensors (PyTorch provides device
memory and streams); host buffers are numpy arrays. The library must have
been built (``paper_2111_01524_gb300.build.build()``); there is no CPU
fallback, and loading fails loudly if the shared library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

VOF_OK, VOF_EINVAL, VOF_ENOMEM, VOF_ECUDA, VOF_ECAPACITY, VOF_ESTATE, VOF_ECFL = range(7)
PREC_FP64, PREC_MIXED = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
FLUX_FMFPA, FLUX_EMFPA, FLUX_NMFPA = 0, 1, 2  # flux polyhedra (Secs. 2.2.2, 2.2.1, 2.2.3)
RECON_LSGIR, RECON_LSFIR = 0, 1  # interface reconstruction (Secs. 2.1.1, 2.1.2)
NB_VERTS = 19  # polyhedron slots per face in vof_get_flux_polyhedra

_lib = None


class VofError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gvof error {status}: {msg}")
        self.status = status


class _Mesh(C.Structure):
    _fields_ = [("n_vert", C.c_int64), ("n_face", C.c_int64), ("n_cell", C.c_int64),
                ("X", C.c_void_p), ("face_ptr", C.c_void_p), ("face_vert", C.c_void_p),
                ("owner", C.c_void_p), ("neighbour", C.c_void_p)]


class _Opt(C.Structure):
    _fields_ = [("eps", C.c_double), ("beta", C.c_double), ("precision", C.c_int32),
                ("flux_polyhedron", C.c_int32), ("reconstruction", C.c_int32),
                ("lsfir_max_iter", C.c_int32), ("lsfir_tol", C.c_double),
                ("poly_capacity", C.c_int32), ("faces_per_warp", C.c_int32)]


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("c", C.c_double * 3),
                ("a", C.c_double * 3), ("r", C.c_double)]


def shape_struct(shape):
    """vof_shape from an inputs.Shape record (kind, c, a, r)."""
    s = _Shape()
    s.kind = int(shape.kind)
    for i in range(3):
        s.c[i] = shape.c[i]
        s.a[i] = shape.a[i]
    s.r = shape.r
    return s


class _Vel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("period", C.c_double),
                ("omega", C.c_double), ("center", C.c_double * 3), ("u0", C.c_double * 3)]


class Stats(C.Structure):
    _fields_ = [("n_interfacial", C.c_int64), ("n_active_faces", C.c_int64),
                ("n_truncations", C.c_int64), ("n_overflow", C.c_int64),
                ("n_degenerate", C.c_int64), ("n_edgeon", C.c_int64),
                ("volume", C.c_double), ("ebound", C.c_double), ("clip_loss", C.c_double),
                ("cutoff_loss", C.c_double), ("boundary_outflow", C.c_double),
                ("n_clipped", C.c_int64), ("n_repaired", C.c_int64), ("n_escaped", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _ServerOpt(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("precision", C.c_int32),
                ("flux_polyhedron", C.c_int32), ("reconstruction", C.c_int32),
                ("max_batch", C.c_int32), ("reserved", C.c_int32 * 2)]


class ServerStats(C.Structure):
    _fields_ = [("n_submitted", C.c_int64), ("n_queued", C.c_int64), ("n_active", C.c_int64),
                ("n_done", C.c_int64), ("cell_steps", C.c_int64), ("device_bytes", C.c_int64),
                ("peak_device_bytes", C.c_int64), ("budget_bytes", C.c_int64),
                ("n_batches", C.c_int64), ("max_active", C.c_int64),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double),
                ("elapsed_s", C.c_double), ("batch_steps", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


def library_path():
    return _build.LIB


def lib():
    """Open libgvof.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"gvof CUDA library not built: {path} is missing "
                               "(run paper_2111_01524_gb300.build.build())")
        L = C.CDLL(path)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.vof_last_error.restype = C.c_char_p
        L.vof_init.argtypes = [vp, vp, vp, C.POINTER(vp)]
        L.vof_batch_create.argtypes = [vp, C.c_int, vp, vp, C.POINTER(vp)]
        L.vof_advect_step.argtypes = [vp, vp, dbl, dbl, vp]
        L.vof_batch_step.argtypes = [vp, vp, vp, vp, vp]
        L.vof_destroy.argtypes = [vp]
        L.vof_destroy.restype = None
        L.vof_set_fraction.argtypes = [vp, vp, i32, vp]
        L.vof_init_fraction.argtypes = [vp, vp, i32, vp]
        L.vof_get_state.argtypes = [vp, vp, i64, C.POINTER(i64), vp]
        L.vof_set_state.argtypes = [vp, vp, i64, vp]
        L.vof_get_fraction.argtypes = [vp, vp, i32, vp]
        L.vof_reconstruct.argtypes = [vp, vp]
        L.vof_advect.argtypes = [vp, vp, dbl, dbl, vp]
        L.vof_step.argtypes = [vp, vp, dbl, dbl, vp]
        L.vof_suggest_dt.argtypes = [vp, vp, dbl, dbl, dbl, C.POINTER(dbl)]
        L.vof_get_planes.argtypes = [vp, vp, i32, vp]
        L.vof_get_tags.argtypes = [vp, vp, vp, vp, i32, vp]
        L.vof_get_face_flux.argtypes = [vp, vp, vp, i32, vp]
        L.vof_get_geometry.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        L.vof_get_neighbors.argtypes = [vp, vp, vp, C.POINTER(i64)]
        L.vof_get_candidates.argtypes = [vp, vp, C.c_int, vp, vp, i64]
        L.vof_get_flux_polyhedra.argtypes = [vp, vp, dbl, dbl, vp, C.c_int, vp, vp]
        L.vof_get_stats.argtypes = [vp, C.POINTER(Stats), vp]
        L.vof_set_timing.argtypes = [vp, C.c_int]
        L.vof_get_timing.argtypes = [vp, vp, vp, C.c_int]
        L.vof_init_batch.argtypes = [vp, C.c_int, vp, C.POINTER(vp)]
        L.vof_batch_offsets.argtypes = [vp, vp, vp, vp, vp]
        L.vof_advect_batch.argtypes = [vp, vp, vp, vp, vp]
        L.vof_step_batch.argtypes = [vp, vp, vp, vp, vp]
        L.vof_suggest_dt_batch.argtypes = [vp, vp, vp, dbl, vp, vp]
        L.vof_graph_capture.argtypes = [vp, C.c_int, vp]
        L.vof_graph_launch.argtypes = [vp, vp, vp, vp, vp]
        L.vof_autotune.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.vof_autotune_ex.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        for name in ("vof_init_batch", "vof_batch_offsets", "vof_advect_batch", "vof_step_batch",
                     "vof_suggest_dt_batch", "vof_graph_capture", "vof_graph_launch",
                     "vof_autotune", "vof_autotune_ex", "vof_batch_create", "vof_advect_step",
                     "vof_batch_step"):
            getattr(L, name).restype = C.c_int
        L.vof_estimate_bytes.argtypes = [vp, C.c_int, vp, C.POINTER(i64)]
        L.vof_server_create.argtypes = [vp, C.POINTER(vp)]
        L.vof_server_submit.argtypes = [vp, vp, vp, vp, i32, dbl, dbl, C.POINTER(i64)]
        L.vof_server_step.argtypes = [vp, C.POINTER(i32)]
        L.vof_server_drain.argtypes = [vp]
        L.vof_server_poll.argtypes = [vp, i64, C.POINTER(i32), vp, C.POINTER(dbl)]
        L.vof_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.vof_server_destroy.argtypes = [vp]
        L.vof_server_destroy.restype = None
        for name in ("vof_estimate_bytes", "vof_server_create", "vof_server_submit",
                     "vof_server_step", "vof_server_drain", "vof_server_poll",
                     "vof_server_get_stats"):
            getattr(L, name).restype = C.c_int
        L.vof_halo_lists.argtypes = [vp, C.c_int, vp, vp]
        L.vof_halo_export.argtypes = [vp, C.c_int, vp, vp]
        L.vof_halo_import.argtypes = [vp, C.c_int, vp, vp]
        L.vof_list_volume.argtypes = [vp, C.c_int, C.POINTER(dbl), vp]
        L.vof_dt_bounds.argtypes = [vp, vp, vp, vp]
        L.vof_dt_from_bounds.argtypes = [vp, vp, vp, dbl, dbl, dbl, C.POINTER(dbl)]
        for name in ("vof_halo_lists", "vof_halo_export", "vof_halo_import", "vof_list_volume",
                     "vof_dt_bounds", "vof_dt_from_bounds"):
            getattr(L, name).restype = C.c_int
        L.vof_volume_sum_noalloc.argtypes = [vp, vp, i64, vp, vp]
        L.vof_volume_sum_noalloc.restype = C.c_int
        L.vof_device_bytes.restype = i64
        L.vof_device_bytes.argtypes = [vp]
        for name in ("vof_init", "vof_set_fraction", "vof_init_fraction", "vof_get_fraction",
                     "vof_reconstruct", "vof_get_state", "vof_set_state",
                     "vof_advect", "vof_step", "vof_suggest_dt", "vof_get_planes",
                     "vof_get_tags", "vof_get_face_flux", "vof_get_geometry",
                     "vof_get_neighbors", "vof_get_candidates", "vof_get_flux_polyhedra",
                     "vof_get_stats", "vof_set_timing", "vof_get_timing"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status):
    if status != VOF_OK:
        raise VofError(status, lib().vof_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _mem(a):
    return MEM_DEVICE if hasattr(a, "data_ptr") and a.is_cuda else MEM_HOST


def dt_from_bounds(vel, hmin, umax, t, cfl, t_end):
    """vof_suggest_dt's time step from per-axis bounds reduced over the parts
    of a partitioned grid (``Context.dt_bounds``)."""
    v = velocity_struct(vel)
    h = np.ascontiguousarray(hmin, np.float64)
    u = np.ascontiguousarray(umax, np.float64)
    if h.shape != (3,) or u.shape != (3,):
        raise ValueError("hmin and umax hold three values each")
    d = C.c_double()
    _check(lib().vof_dt_from_bounds(C.byref(v), _ptr(h), _ptr(u), t, cfl, t_end, C.byref(d)))
    return d.value


def _need_device(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.numel() >= n):
        raise ValueError(f"expected a contiguous CUDA float64 tensor of at least {n} values")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:  # pragma: no cover
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def volume_sum_noalloc(w, F, out, n=None, stream=None):
    """sum_i w[i] * F[i] into out[0] through the allocation-free entry point.

    w, F, out are CUDA tensors (float64) owned by the caller; nothing is
    allocated by the library. Returns the raw status (VOF_OK on success).
    """
    if n is None:
        n = w.numel()
    return lib().vof_volume_sum_noalloc(_ptr(w), _ptr(F), int(n), _ptr(out), _stream(stream))


def estimate_bytes(meshes, precision=PREC_MIXED, flux=FLUX_FMFPA, recon=RECON_LSGIR,
                   poly_capacity=0):
    """Device bytes vof_batch_create would allocate for these meshes (host
    arithmetic on their sizes and connectivity)."""
    meshes = meshes if isinstance(meshes, (list, tuple)) else [meshes]
    keep = []
    descs = (_Mesh * len(meshes))(*[_mesh_desc(m, keep) for m in meshes])
    opt = _Opt()
    opt.eps, opt.beta, opt.precision, opt.flux_polyhedron = 1e-12, 1.5, precision, flux
    opt.reconstruction, opt.poly_capacity = recon, poly_capacity
    out = C.c_int64()
    _check(lib().vof_estimate_bytes(descs, len(meshes), C.byref(opt), C.byref(out)))
    return out.value


class Server:
    """Continuous batching of "advance this interface N steps" requests on
    the device (vof_server_*): requests are admitted, within a device-byte
    budget, as the slots of batched contexts, and every live context advances
    one step per tick."""

    def __init__(self, budget_bytes=0, precision=PREC_MIXED, flux=FLUX_FMFPA, recon=RECON_LSGIR,
                 max_batch=0):
        o = _ServerOpt()
        o.budget_bytes, o.precision, o.flux_polyhedron = int(budget_bytes), precision, flux
        o.reconstruction, o.max_batch = recon, max_batch
        h = C.c_void_p()
        _check(lib().vof_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self.n_cell = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().vof_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, mesh, F0, vel, n_steps, cfl=0.5, t_end=1e9):
        keep = []
        d = _mesh_desc(mesh, keep)
        F0 = np.ascontiguousarray(F0, np.float64)
        v = velocity_struct(vel)
        rid = C.c_int64()
        _check(lib().vof_server_submit(self._h, C.byref(d), _ptr(F0), C.byref(v), int(n_steps),
                                       float(cfl), float(t_end), C.byref(rid)))
        self.n_cell[rid.value] = int(mesh["n_cell"])
        return rid.value

    def step(self):
        n = C.c_int32()
        _check(lib().vof_server_step(self._h, C.byref(n)))
        return n.value

    def drain(self):
        _check(lib().vof_server_drain(self._h))

    def poll(self, rid):
        """(state, F or None, latency_s) of a request"""
        st = C.c_int32()
        lat = C.c_double()
        F = np.empty(self.n_cell[rid])
        _check(lib().vof_server_poll(self._h, int(rid), C.byref(st), _ptr(F), C.byref(lat)))
        return st.value, (F if st.value == REQ_DONE else None), lat.value

    def stats(self):
        s = ServerStats()
        _check(lib().vof_server_get_stats(self._h, C.byref(s)))
        return s.as_dict()


def velocity_struct(v):
    s = _Vel()
    s.kind = v.kind
    s.period = v.period
    s.omega = v.omega
    for i in range(3):
        s.center[i] = v.center[i]
        s.u0[i] = v.u0[i]
    return s


def _mesh_desc(mesh, keep):
    X = np.ascontiguousarray(mesh["X"], np.float64)
    fp = np.ascontiguousarray(mesh["face_ptr"], np.int64)
    fv = np.ascontiguousarray(mesh["face_vert"], np.int32)
    own = np.ascontiguousarray(mesh["owner"], np.int32)
    nbr = np.ascontiguousarray(mesh["neighbour"], np.int32)
    keep.extend([X, fp, fv, own, nbr])
    return _Mesh(X.shape[0], own.shape[0], int(mesh["n_cell"]), _ptr(X).value, _ptr(fp).value,
                 _ptr(fv).value, _ptr(own).value, _ptr(nbr).value)


class Context:
    """Meshes resident on the device with their VOF state (one vof_ctx).

    ``mesh`` is one mesh dict, or a list of them for a batch: the grids are
    joined into one context and advanced together, each with its own
    velocity and time step (the ``*_batch`` methods).
    """

    def __init__(self, mesh, precision=PREC_FP64, eps=1e-12, beta=1.5, flux=FLUX_FMFPA,
                 recon=RECON_LSGIR, lsfir_max_iter=0, lsfir_tol=0.0, poly_capacity=0,
                 faces_per_warp=0, stream=None):
        L = lib()
        meshes = mesh if isinstance(mesh, (list, tuple)) else [mesh]
        keep = []
        descs = (_Mesh * len(meshes))(*[_mesh_desc(m, keep) for m in meshes])
        opt = _Opt()
        opt.eps, opt.beta, opt.precision, opt.flux_polyhedron = eps, beta, precision, flux
        opt.reconstruction, opt.lsfir_max_iter, opt.lsfir_tol = recon, lsfir_max_iter, lsfir_tol
        opt.poly_capacity = poly_capacity
        opt.faces_per_warp = faces_per_warp
        h = C.c_void_p()
        _check(L.vof_batch_create(descs, len(meshes), C.byref(opt), _stream(stream), C.byref(h)))
        self._h = h
        self.n_grids = len(meshes)
        self.n_vert = sum(d.n_vert for d in descs)
        self.n_face = sum(d.n_face for d in descs)
        self.n_cell = sum(d.n_cell for d in descs)
        self.precision = precision
        self.flux = flux
        self.recon = recon
        co = np.empty(self.n_grids + 1, np.int64)
        fo = np.empty(self.n_grids + 1, np.int64)
        vo = np.empty(self.n_grids + 1, np.int64)
        _check(L.vof_batch_offsets(h, None, _ptr(co), _ptr(fo), _ptr(vo)))
        self.cell_off, self.face_off, self.vert_off = co, fo, vo
        del keep  # the host copies are not needed after init

    def close(self):
        if getattr(self, "_h", None):
            lib().vof_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self):
        return lib().vof_device_bytes(self._h)

    # --- state
    def set_fraction(self, F, stream=None):
        if not hasattr(F, "data_ptr"):
            F = np.ascontiguousarray(F, np.float64)
        _check(lib().vof_set_fraction(self._h, _ptr(F), _mem(F), _stream(stream)))

    def init_fraction(self, shape, ndiv=10, stream=None):
        """initfgrid (Sec. 3.2) on the device: F from a body (inputs.Shape)."""
        s = shape_struct(shape)
        _check(lib().vof_init_fraction(self._h, C.byref(s), int(ndiv), _stream(stream)))

    def get_state(self, stream=None):
        """checkpoint: the state a step continues from, as bytes (numpy uint8)"""
        need = C.c_int64()
        _check(lib().vof_get_state(self._h, None, 0, C.byref(need), _stream(stream)))
        buf = np.empty(need.value, np.uint8)
        _check(lib().vof_get_state(self._h, _ptr(buf), buf.size, None, _stream(stream)))
        return buf

    def set_state(self, buf, stream=None):
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().vof_set_state(self._h, _ptr(buf), buf.size, _stream(stream)))

    def get_fraction(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.n_cell)
        _check(lib().vof_get_fraction(self._h, _ptr(out), _mem(out), _stream(stream)))
        return out

    # --- the method
    def reconstruct(self, stream=None):
        _check(lib().vof_reconstruct(self._h, _stream(stream)))

    def advect(self, vel, t, dt, stream=None):
        v = velocity_struct(vel)
        _check(lib().vof_advect_step(self._h, C.byref(v), t, dt, _stream(stream)))

    def step(self, vel, t, dt, stream=None):
        v = velocity_struct(vel)
        _check(lib().vof_step(self._h, C.byref(v), t, dt, _stream(stream)))

    # --- batched forms (one velocity, time and step per grid)
    def _batch_args(self, vels, t, dt):
        vels = list(vels) if isinstance(vels, (list, tuple)) else [vels] * self.n_grids
        va = (_Vel * self.n_grids)(*[velocity_struct(v) for v in vels])
        ta = np.ascontiguousarray(np.broadcast_to(np.asarray(t, np.float64), (self.n_grids,)))
        da = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (self.n_grids,)))
        return va, ta, da

    def advect_batch(self, vels, t, dt, stream=None):
        va, ta, da = self._batch_args(vels, t, dt)
        _check(lib().vof_advect_batch(self._h, va, _ptr(ta), _ptr(da), _stream(stream)))

    def step_batch(self, vels, t, dt, stream=None):
        va, ta, da = self._batch_args(vels, t, dt)
        _check(lib().vof_batch_step(self._h, va, _ptr(ta), _ptr(da), _stream(stream)))

    def suggest_dt_batch(self, vels, t, cfl, t_end):
        va, ta, te = self._batch_args(vels, t, t_end)
        out = np.empty(self.n_grids)
        _check(lib().vof_suggest_dt_batch(self._h, va, _ptr(ta), cfl, _ptr(te), _ptr(out)))
        return out

    def graph_capture(self, with_reconstruct=True, stream=None):
        _check(lib().vof_graph_capture(self._h, 1 if with_reconstruct else 0, _stream(stream)))

    def graph_launch(self, vels, t, dt, stream=None):
        va, ta, da = self._batch_args(vels, t, dt)
        _check(lib().vof_graph_launch(self._h, va, _ptr(ta), _ptr(da), _stream(stream)))

    def autotune(self, vels, t, dt, stream=None, full=False):
        """The tuned launch shape: (flux blocks, reconstruction blocks), and
        with full=True also faces per warp and prebuilt polyhedra (1/0)."""
        va, ta, da = self._batch_args(vels, t, dt)
        fb, rb, fw, pb = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().vof_autotune_ex(self._h, va, _ptr(ta), _ptr(da), _stream(stream), C.byref(fb),
                                     C.byref(rb), C.byref(fw), C.byref(pb)))
        if full:
            return fb.value, rb.value, fw.value, pb.value
        return fb.value, rb.value

    def suggest_dt(self, vel, t, cfl, t_end):
        v = velocity_struct(vel)
        d = C.c_double()
        _check(lib().vof_suggest_dt(self._h, C.byref(v), t, cfl, t_end, C.byref(d)))
        return d.value

    # --- partitioned grids: cell lists, halo gather / scatter, dt bounds
    def set_lists(self, lists):
        """Upload cell lists (a sequence of int arrays of this context's cell
        indices); list k is then addressed by k."""
        lists = [np.ascontiguousarray(a, np.int32).ravel() for a in lists]
        ptr = np.zeros(len(lists) + 1, np.int64)
        for k, a in enumerate(lists):
            ptr[k + 1] = ptr[k] + a.size
        cells = np.concatenate(lists) if lists else np.zeros(1, np.int32)
        cells = np.ascontiguousarray(cells, np.int32)
        _check(lib().vof_halo_lists(self._h, len(lists), _ptr(ptr), _ptr(cells)))
        self._list_sizes = [int(a.size) for a in lists]

    def export_list(self, k, out, stream=None):
        """out (a CUDA float64 tensor of the list's size) <- F over list k."""
        _need_device(out, self._list_sizes[k])
        _check(lib().vof_halo_export(self._h, int(k), C.c_void_p(out.data_ptr()), _stream(stream)))

    def import_list(self, k, src, stream=None):
        """F over list k <- src (a CUDA float64 tensor of the list's size)."""
        _need_device(src, self._list_sizes[k])
        _check(lib().vof_halo_import(self._h, int(k), C.c_void_p(src.data_ptr()), _stream(stream)))

    def list_volume(self, k, stream=None):
        v = C.c_double()
        _check(lib().vof_list_volume(self._h, int(k), C.byref(v), _stream(stream)))
        return v.value

    def dt_bounds(self, vel):
        """(hmin[3], umax[3]) of this grid for the field ``vel``."""
        v = velocity_struct(vel)
        h = np.empty(3)
        u = np.empty(3)
        _check(lib().vof_dt_bounds(self._h, C.byref(v), _ptr(h), _ptr(u)))
        return h, u

    # --- read-back
    def planes(self, stream=None):
        out = np.empty((self.n_cell, 4))
        _check(lib().vof_get_planes(self._h, _ptr(out), MEM_HOST, _stream(stream)))
        return out

    def tags(self, stream=None):
        tv = np.empty(self.n_vert, np.int8)
        tf = np.empty(self.n_face, np.int8)
        tc = np.empty(self.n_cell, np.int8)
        _check(lib().vof_get_tags(self._h, _ptr(tv), _ptr(tf), _ptr(tc), MEM_HOST, _stream(stream)))
        return tv, tf, tc

    def face_flux(self, stream=None):
        Vd = np.empty(self.n_face)
        VF = np.empty(self.n_face)
        _check(lib().vof_get_face_flux(self._h, _ptr(Vd), _ptr(VF), MEM_HOST, _stream(stream)))
        return Vd, VF

    def geometry(self, stream=None):
        g = dict(cell_vol=np.empty(self.n_cell), cell_cen=np.empty((self.n_cell, 3)),
                 face_cen=np.empty((self.n_face, 3)), face_nrm=np.empty((self.n_face, 3)),
                 face_area=np.empty(self.n_face))
        _check(lib().vof_get_geometry(self._h, _ptr(g["cell_vol"]), _ptr(g["cell_cen"]),
                                      _ptr(g["face_cen"]), _ptr(g["face_nrm"]),
                                      _ptr(g["face_area"]), MEM_HOST, _stream(stream)))
        return g

    def neighbors(self):
        n = C.c_int64()
        _check(lib().vof_get_neighbors(self._h, None, None, C.byref(n)))
        ptr = np.empty(self.n_cell + 1, np.int64)
        idx = np.empty(max(n.value, 1), np.int32)
        _check(lib().vof_get_neighbors(self._h, _ptr(ptr), _ptr(idx), C.byref(n)))
        return ptr, idx[:n.value]

    def candidates(self, faces):
        faces = np.ascontiguousarray(faces, np.int32)
        ptr = np.empty(len(faces) + 1, np.int64)
        _check(lib().vof_get_candidates(self._h, _ptr(faces), len(faces), _ptr(ptr), None, 0))
        idx = np.empty(max(int(ptr[-1]), 1), np.int32)
        _check(lib().vof_get_candidates(self._h, _ptr(faces), len(faces), _ptr(ptr), _ptr(idx),
                                        idx.shape[0]))
        return [idx[ptr[i]:ptr[i + 1]].copy() for i in range(len(faces))]

    def flux_polyhedra(self, vel, t, dt, faces):
        faces = np.ascontiguousarray(faces, np.int32)
        verts = np.zeros((len(faces), NB_VERTS, 3))
        counts = np.empty(len(faces), np.int32)
        v = velocity_struct(vel)
        _check(lib().vof_get_flux_polyhedra(self._h, C.byref(v), t, dt, _ptr(faces), len(faces),
                                            _ptr(verts), _ptr(counts)))
        def npts(nI):  # 3I+1 (EMFPA), 2I (NMFPA), 2I+1 (FMFPA)
            return 3 * nI + 1 if self.flux == FLUX_EMFPA else 2 * nI + (self.flux != FLUX_NMFPA)
        return [verts[i, :npts(counts[i])].copy() if counts[i] > 0 else None
                for i in range(len(faces))]

    PHASES = ("cell_tags", "node_tags", "reconstruct", "face_sweep", "flux", "update", "polyhedra",
              "repair")

    def set_timing(self, on=True):
        _check(lib().vof_set_timing(self._h, 1 if on else 0))

    def timing(self):
        """Accumulated per-phase device milliseconds and launch counts since
        the last call (CUDA events on the launching stream)."""
        ms = np.zeros(len(self.PHASES))
        n = np.zeros(len(self.PHASES), np.int64)
        _check(lib().vof_get_timing(self._h, _ptr(ms), _ptr(n), len(self.PHASES)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PHASES)}

    def stats(self, stream=None, raise_on_escape=False):
        """Counters and sums of the last advect. VOF_ECFL (flux polyhedra
        left their candidate cells) is reported as ``cfl_escape`` and raised
        only when asked."""
        s = Stats()
        st = lib().vof_get_stats(self._h, C.byref(s), _stream(stream))
        if st != VOF_ECFL or raise_on_escape:
            _check(st)
        d = s.as_dict()
        d["cfl_escape"] = st == VOF_ECFL
        return d

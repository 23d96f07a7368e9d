// Shared declarations of the gvof CUDA library: device views of the mesh and
// state, the context, velocity evaluation, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/vof.h"

#define GVOF_FULL 0xffffffffu

namespace gvof {

constexpr int kSMs = 152;  // GB300
constexpr int kMaxFaceVerts = 8;

// device view of the mesh: every array is SoA so that per-face and
// per-cell sweeps load coalesced
struct DevMesh {
  int64_t nv, nf, nc;
  const double *x, *y, *z;
  const int64_t* fptr;
  const int32_t* fvert;
  const int32_t* own;
  const int32_t* nbr;
  const double *fcx, *fcy, *fcz;  // face area centroid
  const double *fnx, *fny, *fnz;  // unit normal out of the owner
  const double* fa;               // face area
  const int64_t* cf_ptr;          // cell -> faces; entry f >= 0: owner side, ~f: neighbour side
  const int32_t* cf;
  const int64_t* cv_ptr;          // cell -> vertices (ascending)
  const int32_t* cv;
  const int64_t* vc_ptr;          // vertex -> cells (ascending)
  const int32_t* vc;
  const int64_t* nb_ptr;          // neigbcell (ascending, self excluded)
  const int32_t* nb;
  const double *ccx, *ccy, *ccz;  // cell centroid
  const double* cvol;
  const double* bb;               // bounding boxes, SoA: bb[d*nc + c], d = 0..5 (lo xyz, hi xyz)
};

struct DevState {
  double* F;
  double *nx, *ny, *nz, *C;  // PLIC planes
  int8_t *tv, *tf, *tc;      // node / face / cell tags
  double *Vd, *VF;           // face volumes of the last advect
  double* srate;             // (u0(x_f).n_f) A_f of the current velocity field
  int32_t* icells;           // compacted interfacial cells
  int32_t* afaces;           // compacted active faces
  unsigned long long* cnt;   // counters, see Cnt
  double* red;               // reduction scratch [kRedSlots]
};

enum Cnt {
  kNIcells = 0,
  kNAfaces = 1,
  kNTrunc = 2,
  kNOverflow = 3,
  kNDegen = 4,
  kNEdgeOn = 5,
  kUmax = 6,  // 3 slots: max |u0| per axis (bit pattern of non-negative doubles)
  kNCnt = 16
};
constexpr int kRedSlots = 2 * 1024;

struct Vel {
  int kind;
  double period, omega, cx, cy, cz, ux, uy, uz;
};

// velocity of the test problems without its time factor: u(x, t) = g(t) u0(x)
template <typename T>
__device__ __forceinline__ void vel0(const Vel& v, T x, T y, T z, T& u, T& w, T& s);

template <>
__device__ __forceinline__ void vel0<double>(const Vel& v, double x, double y, double z, double& u,
                                             double& w, double& s) {
  if (v.kind == VOF_VEL_DEFORMATION) {
    double sx, cx, sy, cy, sz, cz;
    sincospi(x, &sx, &cx);
    sincospi(y, &sy, &cy);
    sincospi(z, &sz, &cz);
    double s2x = 2.0 * sx * cx, s2y = 2.0 * sy * cy, s2z = 2.0 * sz * cz;
    u = 2.0 * sx * sx * s2y * s2z;
    w = -s2x * sy * sy * s2z;
    s = -s2x * s2y * sz * sz;
  } else if (v.kind == VOF_VEL_ROTATION) {
    u = -v.omega * (y - v.cy);
    w = v.omega * (x - v.cx);
    s = 0.0;
  } else {
    u = v.ux;
    w = v.uy;
    s = v.uz;
  }
}

template <>
__device__ __forceinline__ void vel0<float>(const Vel& v, float x, float y, float z, float& u,
                                            float& w, float& s) {
  if (v.kind == VOF_VEL_DEFORMATION) {
    float sx, cx, sy, cy, sz, cz;
    sincospif(x, &sx, &cx);
    sincospif(y, &sy, &cy);
    sincospif(z, &sz, &cz);
    float s2x = 2.0f * sx * cx, s2y = 2.0f * sy * cy, s2z = 2.0f * sz * cz;
    u = 2.0f * sx * sx * s2y * s2z;
    w = -s2x * sy * sy * s2z;
    s = -s2x * s2y * sz * sz;
  } else if (v.kind == VOF_VEL_ROTATION) {
    u = (float)(-v.omega) * (y - (float)v.cy);
    w = (float)v.omega * (x - (float)v.cx);
    s = 0.0f;
  } else {
    u = (float)v.ux;
    w = (float)v.uy;
    s = (float)v.uz;
  }
}

}  // namespace gvof

struct vof_ctx {
  int64_t nv, nf, nc;
  int64_t nfv, ncf, ncv, nvc, nnb;
  vof_options opt;
  int device;
  // mesh (device)
  double *x, *y, *z;
  int64_t* fptr;
  int32_t* fvert;
  int32_t *own, *nbr;
  double *fcx, *fcy, *fcz, *fnx, *fny, *fnz, *fa;
  int64_t* cf_ptr;
  int32_t* cf;
  int64_t* cv_ptr;
  int32_t* cv;
  int64_t* vc_ptr;
  int32_t* vc;
  int64_t* nb_ptr;
  int32_t* nb;
  double *ccx, *ccy, *ccz, *cvol;
  double* bb;
  uint8_t* convex;
  // state (device)
  double* F;
  double *nx, *ny, *nz, *C;
  int8_t *tv, *tf, *tc;
  double *Vd, *VF, *srate;
  int32_t *icells, *afaces;
  unsigned long long* cnt;
  double* red;
  // host-side caches
  double hmin[3];
  double umax0[3];
  gvof::Vel vel_cached;
  bool vel_valid;
  bool recon_valid;
  int max_face_verts;
  int max_cell_faces;
  int max_cell_verts;
  int64_t bytes;
  void* pinned;  // small pinned host buffer for counters / sums
  // optional per-phase timing (events recorded around each launch)
  bool timing;
  int n_ev_pairs;
  cudaEvent_t ev[2 * 256];
  int ev_phase[256];
  double phase_ms[8];
  int64_t phase_n[8];
};

namespace gvof {

inline DevMesh mesh_view(const vof_ctx* c) {
  DevMesh m;
  m.nv = c->nv; m.nf = c->nf; m.nc = c->nc;
  m.x = c->x; m.y = c->y; m.z = c->z;
  m.fptr = c->fptr; m.fvert = c->fvert; m.own = c->own; m.nbr = c->nbr;
  m.fcx = c->fcx; m.fcy = c->fcy; m.fcz = c->fcz;
  m.fnx = c->fnx; m.fny = c->fny; m.fnz = c->fnz; m.fa = c->fa;
  m.cf_ptr = c->cf_ptr; m.cf = c->cf; m.cv_ptr = c->cv_ptr; m.cv = c->cv;
  m.vc_ptr = c->vc_ptr; m.vc = c->vc; m.nb_ptr = c->nb_ptr; m.nb = c->nb;
  m.ccx = c->ccx; m.ccy = c->ccy; m.ccz = c->ccz; m.cvol = c->cvol; m.bb = c->bb;
  return m;
}

inline DevState state_view(const vof_ctx* c) {
  DevState s;
  s.F = c->F; s.nx = c->nx; s.ny = c->ny; s.nz = c->nz; s.C = c->C;
  s.tv = c->tv; s.tf = c->tf; s.tc = c->tc; s.Vd = c->Vd; s.VF = c->VF; s.srate = c->srate;
  s.icells = c->icells; s.afaces = c->afaces; s.cnt = c->cnt; s.red = c->red;
  return s;
}

inline Vel to_vel(const vof_velocity& v) {
  Vel r;
  r.kind = v.kind; r.period = v.period; r.omega = v.omega;
  r.cx = v.center[0]; r.cy = v.center[1]; r.cz = v.center[2];
  r.ux = v.u0[0]; r.uy = v.u0[1]; r.uz = v.u0[2];
  return r;
}

// time factor g(t) of the separable fields u(x, t) = g(t) u0(x)
inline double time_factor(const Vel& v, double t) {
  if (v.kind == VOF_VEL_DEFORMATION) return std::cos(3.14159265358979323846 * t / v.period);
  return 1.0;
}

// ------------------------------------------------------------ launchers
// set-up (k_setup.cu)
cudaError_t launch_face_geometry(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_cell_geometry(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_velocity_setup(const vof_ctx* c, const Vel& v, cudaStream_t s);
// sweeps (k_sweep.cu)
cudaError_t launch_cell_tags(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_node_tags(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_face_sweep(const vof_ctx* c, double g_half, double dt, cudaStream_t s);
cudaError_t launch_update(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_volume_sum(const vof_ctx* c, cudaStream_t s);  // writes red[0], red[1]
// reconstruction (k_recon.cu)
cudaError_t launch_reconstruct(const vof_ctx* c, cudaStream_t s);
// flux (k_flux.cu)
cudaError_t launch_flux(const vof_ctx* c, const Vel& v, double g_half, double dt, cudaStream_t s);
cudaError_t launch_candidates(const vof_ctx* c, const int32_t* faces, int n, int64_t cap_per_face,
                              int32_t* out, int32_t* counts, cudaStream_t s);
cudaError_t launch_polyhedra(const vof_ctx* c, const Vel& v, double g_half, double dt,
                             const int32_t* faces, int n, double* verts, int32_t* counts,
                             cudaStream_t s);

}  // namespace gvof

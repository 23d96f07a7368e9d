// C-ABI entry points of the gvof library (declared in include/vof.h).
#include <stdio.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mesh_host.h"
#include "vof_common.cuh"

using namespace gvof;

namespace {

thread_local std::string g_err;
constexpr int kRing = 16;  // pinned slots for per-step grid parameters

vof_status fail(vof_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(VOF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

template <typename T>
cudaError_t dalloc(vof_ctx* c, T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)n);
  if (e == cudaSuccess) c->bytes += (int64_t)(sizeof(T) * (size_t)n);
  return e;
}

void free_all(vof_ctx* c) {
  void* ptrs[] = {c->x, c->y, c->z, c->fptr, c->fvert, c->own, c->nbr, c->fcx, c->fcy, c->fcz,
                  c->fnx, c->fny, c->fnz, c->fa, c->cf_ptr, c->cf, c->cv_ptr, c->cv, c->vc_ptr,
                  c->vc, c->nb_ptr, c->nb, c->ccx, c->ccy, c->ccz, c->cvol, c->bb, c->convex,
                  c->F, c->nx, c->ny, c->nz, c->C, c->tv, c->tf, c->tc, c->Vd, c->VF, c->srate,
                  c->icells, c->afaces, c->cnt, c->red, c->vx2, c->vy2, c->vz2, c->fcx2,
                  c->fcy2, c->fcz2, c->ccx2, c->ccy2, c->ccz2, c->bb2, c->fnx32, c->fny32,
                  c->fnz32, c->fa32, c->cvol32, c->nx32, c->ny32, c->nz32, c->C32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* ptrs2[] = {c->cpl32, c->face_off_d, c->gp_d, c->umax_d, c->acc, c->bfaces, c->vf_ptr, c->vf,
                   c->stamp_c, c->stamp_v, c->stamp_f, c->bcells, c->bnodes, c->lxp, c->lyp,
                   c->lzp, c->lxr, c->lyr, c->lzr, c->lnx, c->lny, c->lnz, c->lnx32, c->lny32,
                   c->lnz32, c->lturn, c->fm_v, c->fm_f, c->fm_meta, c->fm_split, c->dombox,
                   c->fexact, c->Fprev, c->risk, c->repf, c->repc, c->stamp_r, c->Eexc,
                   c->Sroom, c->cover8, c->rstar, c->lists, c->list_part, c->fm_cand,
                   c->fm_cinfo};
  for (void* p : ptrs2)
    if (p) cudaFree(p);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->gp_ring) cudaFreeHost(c->gp_ring);
  for (int i = 0; i < kRing; ++i)
    if (c->ring_ev[i]) cudaEventDestroy(c->ring_ev[i]);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  delete c->cell_off; delete c->face_off; delete c->vert_off;
  delete c->hmin_g; delete c->umax_g; delete c->vel_g;
  delete c->list_ptr;
}

cudaMemcpyKind kind_from_dev(int mem) {
  return mem == VOF_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
}

__global__ void k_pack_planes(int64_t nc, const int8_t* tc, const double* nx, const double* ny,
                              const double* nz, const double* C, double* out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    bool i = tc[c] == 0;
    out[4 * c + 0] = i ? nx[c] : 0.0;
    out[4 * c + 1] = i ? ny[c] : 0.0;
    out[4 * c + 2] = i ? nz[c] : 0.0;
    out[4 * c + 3] = i ? C[c] : 0.0;
  }
}

bool same_vel(const Vel& a, const Vel& b) {
  return a.kind == b.kind && a.period == b.period && a.omega == b.omega && a.cx == b.cx &&
         a.cy == b.cy && a.cz == b.cz && a.ux == b.ux && a.uy == b.uy && a.uz == b.uz;
}

vof_status check_velocity(const vof_velocity& v) {
  if (v.kind < VOF_VEL_DEFORMATION || v.kind > VOF_VEL_DEFORMATION2D)
    return fail(VOF_EINVAL, "unknown velocity kind");
  if ((v.kind == VOF_VEL_DEFORMATION || v.kind == VOF_VEL_DEFORMATION2D) && !(v.period > 0))
    return fail(VOF_EINVAL, "deformation period must be > 0");
  return VOF_OK;
}

// write the per-grid parameters of one step into the device table (through a
// pinned ring slot, so the host may prepare the next step while this copy is
// in flight)
vof_status upload_params(vof_ctx* c, const double* t, const double* dt, cudaStream_t s) {
  const int n = c->n_grids;
  const int slot = c->ring_pos;
  c->ring_pos = (c->ring_pos + 1) % kRing;
  CK(cudaEventSynchronize(c->ring_ev[slot]));  // previous use of this slot done
  GridParam* h = c->gp_ring + (size_t)slot * n;
  for (int g = 0; g < n; ++g) {
    const Vel& v = (*c->vel_g)[g];
    const double tt = t ? t[g] : 0.0, d = dt ? dt[g] : 0.0;
    h[g].vel = v;
    h[g].g = time_factor(v, tt + 0.5 * d);
    h[g].dt = d;
    h[g].gdt = h[g].g * d;
    h[g].pad = 0.0;
  }
  CK(cudaMemcpyAsync(c->gp_d, h, sizeof(GridParam) * n, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(c->ring_ev[slot], s));
  return VOF_OK;
}

// per-face flux rates and per-grid speed maxima of the velocity fields
// (recomputed only when a field changes)
vof_status ensure_velocity(vof_ctx* c, const vof_velocity* vels, cudaStream_t s) {
  if (!vels) return fail(VOF_EINVAL, "velocity is NULL");
  const int n = c->n_grids;
  bool same = c->vel_valid;
  for (int g = 0; g < n; ++g) {
    vof_status st = check_velocity(vels[g]);
    if (st != VOF_OK) return st;
    if (same && !same_vel(to_vel(vels[g]), (*c->vel_g)[g])) same = false;
  }
  if (same) return VOF_OK;
  for (int g = 0; g < n; ++g) (*c->vel_g)[g] = to_vel(vels[g]);
  vof_status st = upload_params(c, nullptr, nullptr, s);
  if (st != VOF_OK) return st;
  CK(launch_velocity_setup(c, s));
  std::vector<unsigned long long> h(3 * n);
  CK(cudaMemcpyAsync(h.data(), c->umax_d, sizeof(unsigned long long) * 3 * n,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < 3 * n; ++i) {
    long long bits = (long long)h[i];
    double x;
    std::memcpy(&x, &bits, sizeof x);
    (*c->umax_g)[i] = x;
  }
  c->vel_valid = true;
  return VOF_OK;
}

// record an event pair around one launch when timing is on
struct PhaseTimer {
  vof_ctx* c;
  cudaStream_t s;
  int slot;
  // launches: kernels the phase launches between the two events
  PhaseTimer(vof_ctx* c_, int phase, cudaStream_t s_, int launches = 1) : c(c_), s(s_), slot(-1) {
    if (!c->timing) return;
    if (c->n_ev_pairs >= 256) flush_timing(c);
    slot = c->n_ev_pairs++;
    c->ev_phase[slot] = phase;
    c->ev_n[slot] = launches;
    cudaEventRecord(c->ev[2 * slot], s);
  }
  ~PhaseTimer() {
    if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], s);
  }
  static void flush_timing(vof_ctx* c) {
    for (int i = 0; i < c->n_ev_pairs; ++i) {
      cudaEventSynchronize(c->ev[2 * i + 1]);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]);
      c->phase_ms[c->ev_phase[i]] += ms;
      c->phase_n[c->ev_phase[i]] += c->ev_n[i];
    }
    c->n_ev_pairs = 0;
  }
};

double dt_from(const double hmin[3], const double um[3], double cfl) {
  double dt = 1e300;
  for (int d = 0; d < 3; ++d)
    if (um[d] > 0.0) dt = std::min(dt, hmin[d] / um[d]);
  return dt * cfl;
}

// the time step of Eq. eq:cfl from the smallest cell extents and the
// largest speeds of the spatial field per axis: the CFL step at t, then
// again with the speeds at the end of that step (a time-modulated field),
// cut at t_end
double dt_for(const Vel& v, const double* hmin, const double* u0, double t, double cfl,
              double t_end) {
  double um[3];
  const double g0 = std::fabs(time_factor(v, t));
  for (int d = 0; d < 3; ++d) um[d] = g0 * u0[d];
  double d1 = dt_from(hmin, um, cfl);
  if (t + d1 > t_end) d1 = t_end - t;
  const double g1 = std::fabs(time_factor(v, t + d1));
  for (int d = 0; d < 3; ++d) um[d] = std::max(um[d], g1 * u0[d]);
  const double d2 = dt_from(hmin, um, cfl);
  double r = std::min(d1, d2);
  if (t + r > t_end) r = t_end - t;
  return r;
}

}  // namespace

namespace gvof {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace gvof

extern "C" {

static vof_status advect_launches(vof_ctx* c, cudaStream_t s);
static vof_status reconstruct_launches(vof_ctx* c, cudaStream_t s);

const char* vof_last_error(void) { return g_err.c_str(); }

int64_t vof_device_bytes(const vof_ctx* c) { return c ? c->bytes : 0; }

static vof_status init_impl(const vof_mesh_desc* mesh, const vof_options* opt, cudaStream_t s,
                            vof_ctx** out, const std::vector<int64_t>& cell_off,
                            const std::vector<int64_t>& face_off,
                            const std::vector<int64_t>& vert_off, const HostConn* pre = nullptr) {
  const int64_t nv = mesh->n_vert, nf = mesh->n_face, nc = mesh->n_cell;
  if (nv <= 0 || nf <= 0 || nc <= 0) return fail(VOF_EINVAL, "empty mesh");
  if (nv >= (1LL << 31) || nf >= (1LL << 31) || nc >= (1LL << 31))
    return fail(VOF_EINVAL, "mesh too large for 32-bit indices");
  if (!mesh->X || !mesh->face_ptr || !mesh->face_vert || !mesh->owner || !mesh->neighbour)
    return fail(VOF_EINVAL, "mesh array is NULL");
  if (mesh->face_ptr[0] != 0) return fail(VOF_EINVAL, "face_ptr[0] != 0");
  int maxI = 0;
  for (int64_t f = 0; f < nf; ++f) {
    int64_t I = mesh->face_ptr[f + 1] - mesh->face_ptr[f];
    if (I < 3 || I > kMaxFaceVerts)
      return fail(VOF_EINVAL, "face " + std::to_string(f) + " has " + std::to_string(I) +
                                  " nodes (3..8 supported)");
    maxI = std::max<int>(maxI, (int)I);
    int32_t o = mesh->owner[f], n = mesh->neighbour[f];
    if (o < 0 || o >= nc || n >= nc || n == o)
      return fail(VOF_EINVAL, "face " + std::to_string(f) + ": bad owner/neighbour");
  }
  const int64_t nfv = mesh->face_ptr[nf];
  for (int64_t k = 0; k < nfv; ++k)
    if (mesh->face_vert[k] < 0 || mesh->face_vert[k] >= nv)
      return fail(VOF_EINVAL, "face_vert entry out of range");
  vof_options o;
  if (opt) o = *opt;
  else {
    std::memset(&o, 0, sizeof o);
    o.eps = 1e-12;
    o.beta = 1.5;
    o.precision = VOF_PREC_FP64;
  }
  if (!(o.eps > 0 && o.eps < 0.5) || !(o.beta > 0) ||
      (o.precision != VOF_PREC_FP64 && o.precision != VOF_PREC_MIXED) ||
      (o.flux_polyhedron != VOF_FLUX_FMFPA && o.flux_polyhedron != VOF_FLUX_EMFPA &&
       o.flux_polyhedron != VOF_FLUX_NMFPA) ||
      (o.reconstruction != VOF_RECON_LSGIR && o.reconstruction != VOF_RECON_LSFIR))
    return fail(VOF_EINVAL, "bad options");
  if (o.lsfir_max_iter < 0 || o.lsfir_max_iter > kMaxLsfirIter || !(o.lsfir_tol >= 0.0))
    return fail(VOF_EINVAL, "lsfir_max_iter must be in 0..16 and lsfir_tol >= 0");
  if (o.lsfir_max_iter == 0) o.lsfir_max_iter = 4;  // n_out of Sec. 3.6
  if (o.lsfir_tol == 0.0) o.lsfir_tol = 1e-3;
  if (o.faces_per_warp < 0 || o.faces_per_warp > 2)
    return fail(VOF_EINVAL, "faces_per_warp must be 0, 1 or 2");
  if (o.poly_capacity < 0) return fail(VOF_EINVAL, "poly_capacity must be >= 0");
  if (o.flux_polyhedron == VOF_FLUX_EMFPA && maxI > kMaxEmfpaVerts)
    return fail(VOF_EINVAL, "EMFPA supports faces of at most 6 nodes; this mesh has " +
                                std::to_string(maxI));

  // the derived connectivity, unless the caller built it already
  HostConn built;
  std::string err;
  if (!pre && !build_connectivity(nv, nf, nc, mesh->face_ptr, mesh->face_vert, mesh->owner,
                                  mesh->neighbour, built, err))
    return fail(VOF_EINVAL, err);
  const HostConn& hc = pre ? *pre : built;
  if (hc.max_cell_faces > 32 || hc.max_cell_verts > 32 || hc.max_cell_entries > 128)
    return fail(VOF_EINVAL, "cell too large (<= 32 faces, 32 nodes, 128 face-node entries)");

  vof_ctx* c = new vof_ctx();
  std::memset((void*)c, 0, sizeof(vof_ctx));
  c->nv = nv; c->nf = nf; c->nc = nc; c->nfv = nfv;
  c->ncf = hc.cf_ptr[nc]; c->ncv = hc.cv_ptr[nc]; c->nvc = hc.vc_ptr[nv]; c->nnb = hc.nb_ptr[nc];
  c->opt = o;
  c->max_face_verts = maxI;
  c->max_cell_faces = hc.max_cell_faces;
  c->max_cell_verts = hc.max_cell_verts;
  cudaGetDevice(&c->device);
  const int ng = (int)cell_off.size() - 1;
  c->n_grids = ng;
  c->cell_off = new std::vector<int64_t>(cell_off);
  c->face_off = new std::vector<int64_t>(face_off);
  c->vert_off = new std::vector<int64_t>(vert_off);
  c->hmin_g = new std::vector<double>(3 * ng, 0.0);
  c->umax_g = new std::vector<double>(3 * ng, 0.0);
  c->vel_g = new std::vector<Vel>(ng);
  auto cleanup = [&](vof_status s, const std::string& m) {
    free_all(c);
    delete c;
    return fail(s, m);
  };
#define CKI(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      vof_status s_ = (e_ == cudaErrorMemoryAllocation) ? VOF_ENOMEM : VOF_ECUDA;          \
      return cleanup(s_, std::string(#call) + ": " + cudaGetErrorString(e_));             \
    }                                                                                      \
  } while (0)
  CKI(dalloc(c, &c->x, nv)); CKI(dalloc(c, &c->y, nv)); CKI(dalloc(c, &c->z, nv));
  CKI(dalloc(c, &c->fptr, nf + 1)); CKI(dalloc(c, &c->fvert, nfv));
  CKI(dalloc(c, &c->own, nf)); CKI(dalloc(c, &c->nbr, nf));
  CKI(dalloc(c, &c->fcx, nf)); CKI(dalloc(c, &c->fcy, nf)); CKI(dalloc(c, &c->fcz, nf));
  CKI(dalloc(c, &c->fnx, nf)); CKI(dalloc(c, &c->fny, nf)); CKI(dalloc(c, &c->fnz, nf));
  CKI(dalloc(c, &c->fa, nf));
  CKI(dalloc(c, &c->cf_ptr, nc + 1)); CKI(dalloc(c, &c->cf, c->ncf));
  CKI(dalloc(c, &c->cv_ptr, nc + 1)); CKI(dalloc(c, &c->cv, c->ncv));
  CKI(dalloc(c, &c->vc_ptr, nv + 1)); CKI(dalloc(c, &c->vc, c->nvc));
  CKI(dalloc(c, &c->nb_ptr, nc + 1)); CKI(dalloc(c, &c->nb, c->nnb));
  CKI(dalloc(c, &c->ccx, nc)); CKI(dalloc(c, &c->ccy, nc)); CKI(dalloc(c, &c->ccz, nc));
  CKI(dalloc(c, &c->cvol, nc)); CKI(dalloc(c, &c->bb, 6 * nc)); CKI(dalloc(c, &c->convex, nc));
  CKI(dalloc(c, &c->F, nc));
  CKI(dalloc(c, &c->nx, nc)); CKI(dalloc(c, &c->ny, nc)); CKI(dalloc(c, &c->nz, nc));
  CKI(dalloc(c, &c->C, nc));
  CKI(dalloc(c, &c->tv, nv)); CKI(dalloc(c, &c->tf, nf)); CKI(dalloc(c, &c->tc, nc));
  CKI(dalloc(c, &c->Vd, nf)); CKI(dalloc(c, &c->VF, nf)); CKI(dalloc(c, &c->srate, nf));
  CKI(dalloc(c, &c->icells, nc)); CKI(dalloc(c, &c->afaces, nf));
  CKI(dalloc(c, &c->cnt, kNCnt)); CKI(dalloc(c, &c->red, kRedSlots));
  CKI(dalloc(c, &c->acc, kNAcc * kAccSlots));
  {
    // node -> faces CSR for the band-limited face sweep
    std::vector<int64_t> vp(nv + 1, 0);
    for (int64_t k = 0; k < nfv; ++k) ++vp[mesh->face_vert[k] + 1];
    for (int64_t v = 0; v < nv; ++v) vp[v + 1] += vp[v];
    std::vector<int32_t> vfl(nfv);
    std::vector<int64_t> pos(vp.begin(), vp.end() - 1);
    for (int64_t f = 0; f < nf; ++f)
      for (int64_t k = mesh->face_ptr[f]; k < mesh->face_ptr[f + 1]; ++k)
        vfl[pos[mesh->face_vert[k]]++] = (int32_t)f;
    CKI(dalloc(c, &c->vf_ptr, nv + 1));
    CKI(dalloc(c, &c->vf, nfv));
    CKI(cudaMemcpyAsync(c->vf_ptr, vp.data(), sizeof(int64_t) * (nv + 1), cudaMemcpyHostToDevice, s));
    CKI(cudaMemcpyAsync(c->vf, vfl.data(), sizeof(int32_t) * nfv, cudaMemcpyHostToDevice, s));
    CKI(dalloc(c, &c->stamp_c, nc)); CKI(dalloc(c, &c->stamp_v, nv)); CKI(dalloc(c, &c->stamp_f, nf));
    CKI(dalloc(c, &c->bcells, nc)); CKI(dalloc(c, &c->bnodes, nv));
    CKI(cudaMemsetAsync(c->stamp_c, 0, sizeof(int32_t) * nc, s));
    CKI(cudaMemsetAsync(c->stamp_v, 0, sizeof(int32_t) * nv, s));
    CKI(cudaMemsetAsync(c->stamp_f, 0, sizeof(int32_t) * nf, s));
  }
  {
    std::vector<int32_t> bf;
    for (int64_t f = 0; f < nf; ++f)
      if (mesh->neighbour[f] < 0) bf.push_back((int32_t)f);
    c->nbf = (int64_t)bf.size();
    CKI(dalloc(c, &c->bfaces, c->nbf > 0 ? c->nbf : 1));
    if (c->nbf > 0)
      CKI(cudaMemcpyAsync(c->bfaces, bf.data(), sizeof(int32_t) * c->nbf, cudaMemcpyHostToDevice, s));
  }
  if (o.precision == VOF_PREC_MIXED) {
    CKI(dalloc(c, &c->vx2, nv)); CKI(dalloc(c, &c->vy2, nv)); CKI(dalloc(c, &c->vz2, nv));
    CKI(dalloc(c, &c->fcx2, nf)); CKI(dalloc(c, &c->fcy2, nf)); CKI(dalloc(c, &c->fcz2, nf));
    CKI(dalloc(c, &c->fnx32, nf)); CKI(dalloc(c, &c->fny32, nf)); CKI(dalloc(c, &c->fnz32, nf));
    CKI(dalloc(c, &c->fa32, nf));
    CKI(dalloc(c, &c->ccx2, nc)); CKI(dalloc(c, &c->ccy2, nc)); CKI(dalloc(c, &c->ccz2, nc));
    CKI(dalloc(c, &c->bb2, 6 * nc)); CKI(dalloc(c, &c->cvol32, nc));
    CKI(dalloc(c, &c->nx32, nc)); CKI(dalloc(c, &c->ny32, nc)); CKI(dalloc(c, &c->nz32, nc));
    CKI(dalloc(c, &c->C32, nc));
    CKI(dalloc(c, &c->cpl32, c->ncf));
    // reconciliation of the FP32 face-volume noise at the bounds (k_sweep.cu)
    c->rep_cap = std::min<int64_t>(nf, kFmCap);
    CKI(dalloc(c, &c->fexact, nf)); CKI(dalloc(c, &c->Fprev, nc)); CKI(dalloc(c, &c->risk, nc));
    CKI(dalloc(c, &c->Eexc, nc)); CKI(dalloc(c, &c->Sroom, nc));
    CKI(dalloc(c, &c->repf, c->rep_cap)); CKI(dalloc(c, &c->repc, 2 * c->rep_cap));
    CKI(dalloc(c, &c->stamp_r, nc));
    CKI(cudaMemsetAsync(c->stamp_r, 0, sizeof(int32_t) * nc, s));
    CKI(cudaMemsetAsync(c->fexact, 0, nf, s));
  }
  {
    // bounding box of each grid's domain (flux polyhedron coverage)
    std::vector<double> db(6 * ng);
    for (int g = 0; g < ng; ++g) {
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t v = vert_off[g]; v < vert_off[g + 1]; ++v)
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], mesh->X[3 * v + d]);
          hi[d] = std::max(hi[d], mesh->X[3 * v + d]);
        }
      for (int d = 0; d < 3; ++d) { db[6 * g + d] = lo[d]; db[6 * g + 3 + d] = hi[d]; }
    }
    CKI(dalloc(c, &c->dombox, 6 * ng));
    CKI(cudaMemcpyAsync(c->dombox, db.data(), sizeof(double) * 6 * ng, cudaMemcpyHostToDevice, s));
  }
  {
    // room for the polyhedra the flux kernel reads prebuilt
    c->fm_cap = o.poly_capacity > 0 ? std::min<int64_t>(nf, o.poly_capacity)
                                     : std::min<int64_t>(nf, kFmCap);
    const size_t gs = o.precision == VOF_PREC_MIXED ? sizeof(float) : sizeof(double);
    CKI(cudaMalloc(&c->fm_v, gs * 3 * kFmSlots * c->fm_cap));
    CKI(cudaMalloc(&c->fm_f, gs * 7 * c->fm_cap));
    c->bytes += (int64_t)(gs * (3 * kFmSlots + 7) * c->fm_cap);
    c->fm_use = c->fm_cap;
    CKI(dalloc(c, &c->fm_meta, c->fm_cap));
    CKI(dalloc(c, &c->fm_split, c->fm_cap));
    CKI(dalloc(c, &c->cover8, nf));
    if (cand_lists_on(o, c->nnb, nc)) {
      CKI(dalloc(c, &c->fm_cand, kPreCand * c->fm_cap));
      CKI(dalloc(c, &c->fm_cinfo, c->fm_cap));
    }
  }
  if (o.reconstruction == VOF_RECON_LSFIR) {
    // PLIC centres by cell, accepted normals by band position, max turn per iteration
    if (o.precision == VOF_PREC_MIXED) {
      CKI(dalloc(c, &c->lxr, nc)); CKI(dalloc(c, &c->lyr, nc)); CKI(dalloc(c, &c->lzr, nc));
      CKI(dalloc(c, &c->lnx32, nc)); CKI(dalloc(c, &c->lny32, nc)); CKI(dalloc(c, &c->lnz32, nc));
    } else {
      CKI(dalloc(c, &c->lxp, nc)); CKI(dalloc(c, &c->lyp, nc)); CKI(dalloc(c, &c->lzp, nc));
      CKI(dalloc(c, &c->lnx, nc)); CKI(dalloc(c, &c->lny, nc)); CKI(dalloc(c, &c->lnz, nc));
    }
    CKI(dalloc(c, &c->lturn, kMaxLsfirIter + 1));
  }
  CKI(cudaMallocHost(&c->pinned, 4096));
  CKI(dalloc(c, &c->face_off_d, ng + 1));
  CKI(dalloc(c, &c->gp_d, ng));
  CKI(dalloc(c, &c->umax_d, 3 * ng));
  CKI(cudaMallocHost(&c->gp_ring, sizeof(GridParam) * kRing * ng));
  for (int i = 0; i < kRing; ++i) CKI(cudaEventCreateWithFlags(&c->ring_ev[i], cudaEventDisableTiming));
  CKI(cudaMemcpyAsync(c->face_off_d, face_off.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemsetAsync(c->gp_d, 0, sizeof(GridParam) * ng, s));

  // SoA vertex coordinates
  {
    std::vector<double> t(nv);
    for (int d = 0; d < 3; ++d) {
      for (int64_t v = 0; v < nv; ++v) t[v] = mesh->X[3 * v + d];
      CKI(cudaMemcpyAsync(d == 0 ? c->x : (d == 1 ? c->y : c->z), t.data(), sizeof(double) * nv,
                          cudaMemcpyHostToDevice, s));
    }
  }
  CKI(cudaMemcpyAsync(c->fptr, mesh->face_ptr, sizeof(int64_t) * (nf + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->fvert, mesh->face_vert, sizeof(int32_t) * nfv, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->own, mesh->owner, sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->nbr, mesh->neighbour, sizeof(int32_t) * nf, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->cf_ptr, hc.cf_ptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->cf, hc.cf.data(), sizeof(int32_t) * c->ncf, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->cv_ptr, hc.cv_ptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->cv, hc.cv.data(), sizeof(int32_t) * c->ncv, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->vc_ptr, hc.vc_ptr.data(), sizeof(int64_t) * (nv + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->vc, hc.vc.data(), sizeof(int32_t) * c->nvc, cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->nb_ptr, hc.nb_ptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice, s));
  CKI(cudaMemcpyAsync(c->nb, hc.nb.data(), sizeof(int32_t) * c->nnb, cudaMemcpyHostToDevice, s));
  CKI(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned long long) * kNCnt, s));
  CKI(cudaMemsetAsync(c->red, 0, sizeof(double) * kRedSlots, s));
  CKI(cudaMemsetAsync(c->acc, 0, sizeof(double) * kNAcc * kAccSlots, s));
  CKI(cudaMemsetAsync(c->F, 0, sizeof(double) * nc, s));
  CKI(cudaMemsetAsync(c->nx, 0, sizeof(double) * nc, s));
  CKI(cudaMemsetAsync(c->ny, 0, sizeof(double) * nc, s));
  CKI(cudaMemsetAsync(c->nz, 0, sizeof(double) * nc, s));
  CKI(cudaMemsetAsync(c->C, 0, sizeof(double) * nc, s));
  CKI(cudaMemsetAsync(c->tc, 0xff, nc, s));
  CKI(cudaMemsetAsync(c->Vd, 0, sizeof(double) * nf, s));
  CKI(cudaMemsetAsync(c->VF, 0, sizeof(double) * nf, s));
  CKI(dalloc(c, &c->rstar, nv));
  CKI(launch_face_geometry(c, s));
  CKI(launch_cell_geometry(c, s));
  CKI(launch_node_star(c, s));
  if (o.precision == VOF_PREC_MIXED) CKI(launch_mixed_copies(c, s));
  CKI(cudaStreamSynchronize(s));
  {
    // two faces per warp (a half warp holds at most 16 face loops): an
    // FMFPA polyhedron has up to 3I+1 faces (the cell face, I side quads
    // each split in two, I apex triangles), an NMFPA one I+2; truncation by
    // a convex cell of m faces and the PLIC plane adds at most m+1 more, so
    // base faces + m + 1 <= 16 bounds every loop list the kernel builds
    std::vector<uint8_t> cvx(nc);
    CKI(cudaMemcpy(cvx.data(), c->convex, nc, cudaMemcpyDeviceToHost));
    const int base_faces = o.flux_polyhedron == VOF_FLUX_NMFPA ? maxI + 2 : 3 * maxI + 1;
    bool ok = o.flux_polyhedron != VOF_FLUX_EMFPA && base_faces + hc.max_cell_faces + 1 <= 16;
    for (int64_t k = 0; k < nc && ok; ++k) ok = cvx[k] != 0;
    c->half_ok = ok;
    if (o.faces_per_warp == 2 && !ok)
      return cleanup(VOF_EINVAL, "faces_per_warp = 2 needs FMFPA or NMFPA polyhedra whose faces plus "
                                 "the faces of a convex cell plus one number at most 16");
    c->faces_per_warp = o.faces_per_warp == 0 ? 1 : o.faces_per_warp;
  }
  {
    std::vector<double> bb(6 * nc);
    CKI(cudaMemcpyAsync(bb.data(), c->bb, sizeof(double) * 6 * nc, cudaMemcpyDeviceToHost, s));
    CKI(cudaStreamSynchronize(s));
    for (int g = 0; g < ng; ++g)
      for (int d = 0; d < 3; ++d) {
        double h = 1e300;
        for (int64_t k = cell_off[g]; k < cell_off[g + 1]; ++k)
          h = std::min(h, bb[(3 + d) * nc + k] - bb[d * nc + k]);
        (*c->hmin_g)[3 * g + d] = h;
      }
  }
#undef CKI
  *out = c;
  return VOF_OK;
}

vof_status vof_init(const vof_mesh_desc* mesh, const vof_options* opt, void* stream,
                    vof_ctx** out) {
  if (!mesh || !out) return fail(VOF_EINVAL, "mesh or out is NULL");
  *out = nullptr;
  std::vector<int64_t> co = {0, mesh->n_cell}, fo = {0, mesh->n_face}, vo = {0, mesh->n_vert};
  return init_impl(mesh, opt, (cudaStream_t)stream, out, co, fo, vo);
}

static vof_status batch_create_impl(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                                    void* stream, vof_ctx** out, const HostConn* const* conns);

vof_status vof_batch_create(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                            void* stream, vof_ctx** out) {
  return batch_create_impl(meshes, n_grids, opt, stream, out, nullptr);
}

static vof_status batch_create_impl(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                                    void* stream, vof_ctx** out, const HostConn* const* conns) {
  if (!meshes || !out || n_grids < 1) return fail(VOF_EINVAL, "bad batch arguments");
  *out = nullptr;
  if (n_grids == 1) {
    if (!conns) return vof_init(meshes, opt, stream, out);
    const std::vector<int64_t> co{0, meshes[0].n_cell}, fo{0, meshes[0].n_face},
        vo{0, meshes[0].n_vert};
    return init_impl(meshes, opt, (cudaStream_t)stream, out, co, fo, vo, conns[0]);
  }
  std::vector<int64_t> co(n_grids + 1, 0), fo(n_grids + 1, 0), vo(n_grids + 1, 0), po(n_grids + 1, 0);
  for (int g = 0; g < n_grids; ++g) {
    const vof_mesh_desc& m = meshes[g];
    if (m.n_vert <= 0 || m.n_face <= 0 || m.n_cell <= 0 || !m.X || !m.face_ptr || !m.face_vert ||
        !m.owner || !m.neighbour)
      return fail(VOF_EINVAL, "grid " + std::to_string(g) + ": empty or NULL mesh");
    co[g + 1] = co[g] + m.n_cell;
    fo[g + 1] = fo[g] + m.n_face;
    vo[g + 1] = vo[g] + m.n_vert;
    po[g + 1] = po[g] + m.face_ptr[m.n_face];
  }
  // join the grids: ids of grid g are shifted by the sizes of grids < g
  std::vector<double> X(3 * vo[n_grids]);
  std::vector<int64_t> fp(fo[n_grids] + 1);
  std::vector<int32_t> fv(po[n_grids]), own(fo[n_grids]), nbr(fo[n_grids]);
  for (int g = 0; g < n_grids; ++g) {
    const vof_mesh_desc& m = meshes[g];
    std::memcpy(X.data() + 3 * vo[g], m.X, sizeof(double) * 3 * m.n_vert);
    for (int64_t f = 0; f < m.n_face; ++f) {
      fp[fo[g] + f] = po[g] + m.face_ptr[f];
      own[fo[g] + f] = (int32_t)(m.owner[f] + co[g]);
      nbr[fo[g] + f] = m.neighbour[f] >= 0 ? (int32_t)(m.neighbour[f] + co[g]) : -1;
    }
    for (int64_t k = 0; k < m.face_ptr[m.n_face]; ++k)
      fv[po[g] + k] = (int32_t)(m.face_vert[k] + vo[g]);
  }
  fp[fo[n_grids]] = po[n_grids];
  vof_mesh_desc j;
  j.n_vert = vo[n_grids]; j.n_face = fo[n_grids]; j.n_cell = co[n_grids];
  j.X = X.data(); j.face_ptr = fp.data(); j.face_vert = fv.data(); j.owner = own.data();
  j.neighbour = nbr.data();
  if (!conns) return init_impl(&j, opt, (cudaStream_t)stream, out, co, fo, vo);
  HostConn joined;
  join_connectivity(std::vector<const HostConn*>(conns, conns + n_grids), co, fo, vo, joined);
  return init_impl(&j, opt, (cudaStream_t)stream, out, co, fo, vo, &joined);
}

}  // extern "C"

namespace gvof {
vof_status batch_create_with_conn(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                                  void* stream, vof_ctx** out, const HostConn* const* conns) {
  return batch_create_impl(meshes, n_grids, opt, stream, out, conns);
}
}  // namespace gvof

extern "C" {

vof_status vof_init_batch(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                          vof_ctx** out) {
  return vof_batch_create(meshes, n_grids, opt, nullptr, out);
}

vof_status vof_batch_offsets(vof_ctx* c, int* n_grids, int64_t* cell_off, int64_t* face_off,
                             int64_t* vert_off) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (n_grids) *n_grids = c->n_grids;
  for (int g = 0; g <= c->n_grids; ++g) {
    if (cell_off) cell_off[g] = (*c->cell_off)[g];
    if (face_off) face_off[g] = (*c->face_off)[g];
    if (vert_off) vert_off[g] = (*c->vert_off)[g];
  }
  return VOF_OK;
}

vof_status vof_set_timing(vof_ctx* c, int on) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (on && !c->timing) {
    for (int i = 0; i < 2 * 256; ++i) CK(cudaEventCreate(&c->ev[i]));
    c->n_ev_pairs = 0;
    for (int i = 0; i < 8; ++i) { c->phase_ms[i] = 0; c->phase_n[i] = 0; }
    c->timing = true;
  } else if (!on && c->timing) {
    PhaseTimer::flush_timing(c);
    for (int i = 0; i < 2 * 256; ++i) cudaEventDestroy(c->ev[i]);
    c->timing = false;
  }
  return VOF_OK;
}

vof_status vof_get_timing(vof_ctx* c, double* ms, int64_t* launches, int n) {
  if (!c || n < 0 || n > VOF_NUM_PHASES) return fail(VOF_EINVAL, "bad argument");
  if (c->timing) PhaseTimer::flush_timing(c);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = c->phase_ms[i];
    if (launches) launches[i] = c->phase_n[i];
    c->phase_ms[i] = 0;
    c->phase_n[i] = 0;
  }
  return VOF_OK;
}

void vof_destroy(vof_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->timing) vof_set_timing(c, 0);
  free_all(c);
  delete c;
}

vof_status vof_set_fraction(vof_ctx* c, const double* F, int mem, void* stream) {
  if (!c || !F) return fail(VOF_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  // host values come in through the face-volume export buffer (n_face >= 2
  // n_cell for any closed mesh; scratch between steps)
  const double* src = F;
  if (mem != VOF_MEM_DEVICE) {
    if (c->nf < c->nc) return fail(VOF_EINVAL, "mesh has fewer faces than cells");
    CK(cudaMemcpyAsync(c->Vd, F, sizeof(double) * c->nc, cudaMemcpyHostToDevice, s));
    src = c->Vd;
  }
  // the next sweeps stay band-limited if only band cells of the last advect
  // change, else they are full; the volume bookkeeping starts from this F
  CK(launch_set_fraction(c, src, s));
  CK(cudaMemsetAsync(c->acc, 0, sizeof(double) * kNAcc * kAccSlots, s));
  if (mem != VOF_MEM_DEVICE) CK(cudaStreamSynchronize(s));
  c->recon_valid = false;
  return VOF_OK;
}

vof_status vof_init_fraction(vof_ctx* c, const vof_shape* shape, int ndiv, void* stream) {
  if (!c || !shape) return fail(VOF_EINVAL, "NULL argument");
  if (shape->kind != VOF_SHAPE_SPHERE && shape->kind != VOF_SHAPE_CYLINDER &&
      shape->kind != VOF_SHAPE_HALFSPACE)
    return fail(VOF_EINVAL, "unknown shape kind");
  if (ndiv < 1 || ndiv > 16) return fail(VOF_EINVAL, "ndiv must be in 1..16");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(shape->c[d]) || !std::isfinite(shape->a[d]))
      return fail(VOF_EINVAL, "shape coordinates must be finite");
  if (shape->kind != VOF_SHAPE_SPHERE) {
    const double n = std::sqrt(shape->a[0] * shape->a[0] + shape->a[1] * shape->a[1] +
                               shape->a[2] * shape->a[2]);
    if (!(std::fabs(n - 1.0) <= 1e-12)) return fail(VOF_EINVAL, "shape axis must be a unit vector");
  }
  if (shape->kind != VOF_SHAPE_HALFSPACE && !(shape->r > 0.0 && std::isfinite(shape->r)))
    return fail(VOF_EINVAL, "shape radius must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_init_fraction(c, shape, ndiv, s));
  // as vof_set_fraction: bookkeeping from this F, full sweeps next
  CK(cudaMemsetAsync(c->acc, 0, sizeof(double) * kNAcc * kAccSlots, s));
  CK(cudaMemsetAsync(c->cnt + kBandCellsOk, 0, 2 * sizeof(unsigned long long), s));
  c->recon_valid = false;
  return VOF_OK;
}

vof_status vof_get_fraction(vof_ctx* c, double* F, int mem, void* stream) {
  if (!c || !F) return fail(VOF_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(F, c->F, sizeof(double) * c->nc, kind_from_dev(mem), s));
  if (mem != VOF_MEM_DEVICE) CK(cudaStreamSynchronize(s));
  return VOF_OK;
}

vof_status vof_reconstruct(vof_ctx* c, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  cudaStream_t s = (cudaStream_t)stream;
  vof_status st = reconstruct_launches(c, s);
  if (st != VOF_OK) return st;
  c->recon_valid = true;
  return VOF_OK;
}

static vof_status advect_launches(vof_ctx* c, cudaStream_t s) {
  // launch counts: the kernels each phase launches (band-list kernels included)
  { PhaseTimer tm(c, VOF_PHASE_FACE_SWEEP, s, 2); CK(launch_face_sweep(c, s)); }
  { PhaseTimer tm(c, VOF_PHASE_POLYHEDRA, s, prebuild_lists(c) ? 2 : 1); CK(launch_prebuild(c, s)); }
  { PhaseTimer tm(c, VOF_PHASE_FLUX, s); CK(launch_flux(c, s)); }
  { PhaseTimer tm(c, VOF_PHASE_UPDATE, s, 2); CK(launch_update(c, s)); }
  if (c->opt.precision == VOF_PREC_MIXED) {
    PhaseTimer tm(c, VOF_PHASE_REPAIR, s, repair_launch_count());
    CK(launch_repair(c, s));
  }
  return VOF_OK;
}

static vof_status reconstruct_launches(vof_ctx* c, cudaStream_t s) {
  { PhaseTimer t(c, VOF_PHASE_CELL_TAGS, s); CK(launch_cell_tags(c, s)); }
  { PhaseTimer t(c, VOF_PHASE_NODE_TAGS, s, 3); CK(launch_node_tags(c, s)); }
  { PhaseTimer t(c, VOF_PHASE_RECONSTRUCT, s, reconstruct_launch_count(c)); CK(launch_reconstruct(c, s)); }
  return VOF_OK;
}

static vof_status check_steps(const vof_ctx* c, const double* t, const double* dt) {
  if (!t || !dt) return fail(VOF_EINVAL, "t or dt is NULL");
  for (int g = 0; g < c->n_grids; ++g)
    if (!(dt[g] >= 0) || !std::isfinite(t[g])) return fail(VOF_EINVAL, "dt must be >= 0 and t finite");
  return VOF_OK;
}

vof_status vof_advect_batch(vof_ctx* c, const vof_velocity* vels, const double* t, const double* dt,
                            void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (!c->recon_valid) return fail(VOF_ESTATE, "advect needs a reconstruction of the current F");
  vof_status st = check_steps(c, t, dt);
  if (st != VOF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_velocity(c, vels, s);
  if (st != VOF_OK) return st;
  st = upload_params(c, t, dt, s);
  if (st != VOF_OK) return st;
  st = advect_launches(c, s);
  if (st != VOF_OK) return st;
  c->recon_valid = false;
  return VOF_OK;
}

vof_status vof_step_batch(vof_ctx* c, const vof_velocity* vels, const double* t, const double* dt,
                          void* stream) {
  vof_status st = vof_advect_batch(c, vels, t, dt, stream);
  if (st != VOF_OK) return st;
  return vof_reconstruct(c, stream);
}

vof_status vof_advect(vof_ctx* c, const vof_velocity* vel, double t, double dt, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (c->n_grids != 1) return fail(VOF_EINVAL, "batch context: use vof_advect_batch");
  return vof_advect_batch(c, vel, &t, &dt, stream);
}

vof_status vof_advect_step(vof_ctx* c, const vof_velocity* vel, double t, double dt, void* stream) {
  return vof_advect(c, vel, t, dt, stream);
}

vof_status vof_batch_step(vof_ctx* c, const vof_velocity* vels, const double* t, const double* dt,
                          void* stream) {
  return vof_step_batch(c, vels, t, dt, stream);
}

vof_status vof_step(vof_ctx* c, const vof_velocity* vel, double t, double dt, void* stream) {
  vof_status st = vof_advect(c, vel, t, dt, stream);
  if (st != VOF_OK) return st;
  return vof_reconstruct(c, stream);
}

vof_status vof_suggest_dt_batch(vof_ctx* c, const vof_velocity* vels, const double* t, double cfl,
                                const double* t_end, double* dt_out) {
  if (!c || !t || !t_end || !dt_out) return fail(VOF_EINVAL, "NULL argument");
  if (!(cfl > 0)) return fail(VOF_EINVAL, "cfl must be > 0");
  vof_status st = ensure_velocity(c, vels, 0);
  if (st != VOF_OK) return st;
  for (int gi = 0; gi < c->n_grids; ++gi)
    dt_out[gi] = dt_for((*c->vel_g)[gi], c->hmin_g->data() + 3 * gi, c->umax_g->data() + 3 * gi,
                        t[gi], cfl, t_end[gi]);
  return VOF_OK;
}

vof_status vof_dt_bounds(vof_ctx* c, const vof_velocity* vel, double* hmin, double* umax) {
  if (!c || !vel || !hmin || !umax) return fail(VOF_EINVAL, "NULL argument");
  if (c->n_grids != 1) return fail(VOF_EINVAL, "batch context: one grid only");
  vof_status st = ensure_velocity(c, vel, 0);
  if (st != VOF_OK) return st;
  for (int d = 0; d < 3; ++d) {
    hmin[d] = (*c->hmin_g)[d];
    umax[d] = (*c->umax_g)[d];
  }
  return VOF_OK;
}

vof_status vof_dt_from_bounds(const vof_velocity* vel, const double* hmin, const double* umax,
                              double t, double cfl, double t_end, double* dt) {
  if (!vel || !hmin || !umax || !dt) return fail(VOF_EINVAL, "NULL argument");
  if (!(cfl > 0)) return fail(VOF_EINVAL, "cfl must be > 0");
  vof_status st = check_velocity(*vel);
  if (st != VOF_OK) return st;
  for (int d = 0; d < 3; ++d)
    if (!(hmin[d] > 0.0) || !(umax[d] >= 0.0)) return fail(VOF_EINVAL, "bad bounds");
  *dt = dt_for(to_vel(*vel), hmin, umax, t, cfl, t_end);
  return VOF_OK;
}

vof_status vof_suggest_dt(vof_ctx* c, const vof_velocity* vel, double t, double cfl,
                          double t_end, double* dt) {
  if (!c || !dt) return fail(VOF_EINVAL, "NULL argument");
  if (c->n_grids != 1) return fail(VOF_EINVAL, "batch context: use vof_suggest_dt_batch");
  return vof_suggest_dt_batch(c, vel, &t, cfl, &t_end, dt);
}

vof_status vof_graph_capture(vof_ctx* c, int with_reconstruct, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (c->timing) return fail(VOF_ESTATE, "switch timing off before capturing a graph");
  cudaStream_t s = (cudaStream_t)stream;
  if (s == 0) return fail(VOF_EINVAL, "graph capture needs a non-default stream");
  if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  vof_status st = advect_launches(c, s);
  if (st == VOF_OK && with_reconstruct) st = reconstruct_launches(c, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != VOF_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return fail(VOF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  c->graph = g;
  CK(cudaGraphInstantiate(&c->graph_exec, g, 0));
  c->graph_step = with_reconstruct ? 1 : 0;
  return VOF_OK;
}

vof_status vof_graph_launch(vof_ctx* c, const vof_velocity* vels, const double* t, const double* dt,
                            void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (!c->graph_exec) return fail(VOF_ESTATE, "no captured graph (vof_graph_capture)");
  if (!c->recon_valid) return fail(VOF_ESTATE, "advect needs a reconstruction of the current F");
  vof_status st = check_steps(c, t, dt);
  if (st != VOF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_velocity(c, vels, s);
  if (st != VOF_OK) return st;
  st = upload_params(c, t, dt, s);
  if (st != VOF_OK) return st;
  CK(cudaGraphLaunch(c->graph_exec, s));
  c->recon_valid = c->graph_step == 1;
  return VOF_OK;
}

vof_status vof_autotune_ex(vof_ctx* c, const vof_velocity* vels, const double* t,
                           const double* dt, void* stream, int* flux_blocks, int* recon_blocks,
                           int* faces_per_warp, int* prebuilt) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (!c->recon_valid) return fail(VOF_ESTATE, "autotune needs a reconstruction of the current F");
  vof_status st = check_steps(c, t, dt);
  if (st != VOF_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = ensure_velocity(c, vels, s);
  if (st != VOF_OK) return st;
  st = upload_params(c, t, dt, s);
  if (st != VOF_OK) return st;
  const bool timing = c->timing;
  c->timing = false;
  CK(launch_face_sweep(c, s));  // active faces of the current state (F is not changed)
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int cand[] = {kSMs * 2, kSMs * 4, kSMs * 6, kSMs * 8, kSMs * 12, kSMs * 16};
  // the flux phase: faces per warp x polyhedra prebuilt (their
  // construction timed with the truncations) or built in the flux kernel
  // x blocks; then the reconstruction's blocks
  const int64_t fm_alloc = c->fm_cap;
  float best_f = 1e30f, best_r = 1e30f;
  int bf = kSMs * 8, br = kSMs * 8, bw = 1, bp = 1;
  for (int fpw = 1; fpw <= (c->half_ok ? 2 : 1); ++fpw)
    for (int pb = 1; pb >= 0; --pb)
      for (int g : cand) {
        c->faces_per_warp = fpw;
        c->fm_use = pb ? fm_alloc : 0;
        c->flux_blocks = g;
        float tot = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
          CK(cudaEventRecord(e0, s));
          CK(launch_prebuild(c, s));
          CK(launch_flux(c, s));
          CK(cudaEventRecord(e1, s));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          if (rep > 0) tot += ms;  // first launch warms caches
        }
        if (tot < best_f) { best_f = tot; bf = g; bw = fpw; bp = pb; }
      }
  c->faces_per_warp = bw;
  c->fm_use = bp ? fm_alloc : 0;
  c->flux_blocks = bf;
  for (int g : cand) {
    c->recon_blocks = g;
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0, s));
      CK(launch_reconstruct(c, s));
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) tot += ms;
    }
    if (tot < best_r) { best_r = tot; br = g; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->recon_blocks = br;
  c->timing = timing;
  if (flux_blocks) *flux_blocks = bf;
  if (recon_blocks) *recon_blocks = br;
  if (faces_per_warp) *faces_per_warp = bw;
  if (prebuilt) *prebuilt = bp;
  return VOF_OK;
}

vof_status vof_autotune(vof_ctx* c, const vof_velocity* vels, const double* t, const double* dt,
                        void* stream, int* flux_blocks, int* recon_blocks) {
  return vof_autotune_ex(c, vels, t, dt, stream, flux_blocks, recon_blocks, nullptr, nullptr);
}

namespace {
constexpr uint64_t kStateMagic = 0x45544154534f5647ull;  // "GVOSTATE"
struct StateHeader {
  uint64_t magic;
  int64_t version, nc, nv, nacc;
};
int64_t state_bytes(const vof_ctx* c) {
  return (int64_t)sizeof(StateHeader) + 5 * 8 * c->nc + c->nc + c->nv + 8 * (int64_t)kNAcc * kAccSlots;
}
__global__ void k_planes32(int64_t nc, const double* nx, const double* ny, const double* nz,
                           const double* C, float* nx32, float* ny32, float* nz32, float* C32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    nx32[i] = (float)nx[i]; ny32[i] = (float)ny[i]; nz32[i] = (float)nz[i]; C32[i] = (float)C[i];
  }
}
}  // namespace

vof_status vof_get_state(vof_ctx* c, void* buf, int64_t bytes, int64_t* need, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  const int64_t n = state_bytes(c);
  if (need) *need = n;
  if (!buf) return VOF_OK;
  if (bytes < n) return fail(VOF_EINVAL, "state buffer too small");
  if (!c->recon_valid) return fail(VOF_ESTATE, "the state is taken after a reconstruction");
  cudaStream_t s = (cudaStream_t)stream;
  StateHeader h{kStateMagic, 1, c->nc, c->nv, (int64_t)kNAcc * kAccSlots};
  char* p = (char*)buf;
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  const size_t d = sizeof(double) * c->nc;
  for (const double* a : {c->F, c->nx, c->ny, c->nz, c->C}) {
    CK(cudaMemcpyAsync(p, a, d, cudaMemcpyDeviceToHost, s));
    p += d;
  }
  CK(cudaMemcpyAsync(p, c->tc, c->nc, cudaMemcpyDeviceToHost, s));
  p += c->nc;
  CK(cudaMemcpyAsync(p, c->tv, c->nv, cudaMemcpyDeviceToHost, s));
  p += c->nv;
  CK(cudaMemcpyAsync(p, c->acc, sizeof(double) * kNAcc * kAccSlots, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return VOF_OK;
}

vof_status vof_set_state(vof_ctx* c, const void* buf, int64_t bytes, void* stream) {
  if (!c || !buf) return fail(VOF_EINVAL, "NULL argument");
  const int64_t n = state_bytes(c);
  StateHeader h;
  if (bytes < (int64_t)sizeof h) return fail(VOF_EINVAL, "state buffer too small");
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.version != 1) return fail(VOF_EINVAL, "not a saved state");
  if (h.nc != c->nc || h.nv != c->nv || h.nacc != (int64_t)kNAcc * kAccSlots)
    return fail(VOF_EINVAL, "the state was saved from another mesh");
  if (bytes < n) return fail(VOF_EINVAL, "state buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  const char* p = (const char*)buf + sizeof h;
  const size_t d = sizeof(double) * c->nc;
  for (double* a : {c->F, c->nx, c->ny, c->nz, c->C}) {
    CK(cudaMemcpyAsync(a, p, d, cudaMemcpyHostToDevice, s));
    p += d;
  }
  CK(cudaMemcpyAsync(c->tc, p, c->nc, cudaMemcpyHostToDevice, s));
  p += c->nc;
  CK(cudaMemcpyAsync(c->tv, p, c->nv, cudaMemcpyHostToDevice, s));
  p += c->nv;
  CK(cudaMemcpyAsync(c->acc, p, sizeof(double) * kNAcc * kAccSlots, cudaMemcpyHostToDevice, s));
  // the FP32 planes are the FP64 ones rounded (so stored); band lists are
  // rebuilt by full sweeps
  if (c->opt.precision == VOF_PREC_MIXED) {
    k_planes32<<<kSMs * 4, 256, 0, s>>>(c->nc, c->nx, c->ny, c->nz, c->C, c->nx32, c->ny32, c->nz32,
                                        c->C32);
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(c->cnt + kBandCellsOk, 0, 2 * sizeof(unsigned long long), s));
  CK(cudaStreamSynchronize(s));
  c->recon_valid = true;
  return VOF_OK;
}

vof_status vof_get_planes(vof_ctx* c, double* planes, int mem, void* stream) {
  if (!c || !planes) return fail(VOF_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* dst = planes;
  if (mem != VOF_MEM_DEVICE) CK(cudaMallocAsync((void**)&dst, sizeof(double) * 4 * c->nc, s));
  k_pack_planes<<<kSMs * 8, 256, 0, s>>>(c->nc, c->tc, c->nx, c->ny, c->nz, c->C, dst);
  CK(cudaGetLastError());
  if (mem != VOF_MEM_DEVICE) {
    CK(cudaMemcpyAsync(planes, dst, sizeof(double) * 4 * c->nc, cudaMemcpyDeviceToHost, s));
    CK(cudaFreeAsync(dst, s));
    CK(cudaStreamSynchronize(s));
  }
  return VOF_OK;
}

vof_status vof_get_tags(vof_ctx* c, int8_t* tv, int8_t* tf, int8_t* tc, int mem, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  cudaStream_t s = (cudaStream_t)stream;
  if (tv) CK(cudaMemcpyAsync(tv, c->tv, c->nv, kind_from_dev(mem), s));
  if (tf) CK(cudaMemcpyAsync(tf, c->tf, c->nf, kind_from_dev(mem), s));
  if (tc) CK(cudaMemcpyAsync(tc, c->tc, c->nc, kind_from_dev(mem), s));
  if (mem != VOF_MEM_DEVICE) CK(cudaStreamSynchronize(s));
  return VOF_OK;
}

vof_status vof_get_face_flux(vof_ctx* c, double* Vd, double* VF, int mem, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_face_flux_export(c, s));
  if (Vd) CK(cudaMemcpyAsync(Vd, c->Vd, sizeof(double) * c->nf, kind_from_dev(mem), s));
  if (VF) CK(cudaMemcpyAsync(VF, c->VF, sizeof(double) * c->nf, kind_from_dev(mem), s));
  if (mem != VOF_MEM_DEVICE) CK(cudaStreamSynchronize(s));
  return VOF_OK;
}

vof_status vof_get_geometry(vof_ctx* c, double* cell_vol, double* cell_cen, double* face_cen,
                            double* face_nrm, double* face_area, int mem, void* stream) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyKind k = kind_from_dev(mem);
  if (cell_vol) CK(cudaMemcpyAsync(cell_vol, c->cvol, sizeof(double) * c->nc, k, s));
  if (face_area) CK(cudaMemcpyAsync(face_area, c->fa, sizeof(double) * c->nf, k, s));
  const double* cc[3] = {c->ccx, c->ccy, c->ccz};
  const double* fc[3] = {c->fcx, c->fcy, c->fcz};
  const double* fn[3] = {c->fnx, c->fny, c->fnz};
  for (int d = 0; d < 3; ++d) {
    if (cell_cen)
      CK(cudaMemcpy2DAsync(cell_cen + d, 3 * sizeof(double), cc[d], sizeof(double), sizeof(double),
                           c->nc, k, s));
    if (face_cen)
      CK(cudaMemcpy2DAsync(face_cen + d, 3 * sizeof(double), fc[d], sizeof(double), sizeof(double),
                           c->nf, k, s));
    if (face_nrm)
      CK(cudaMemcpy2DAsync(face_nrm + d, 3 * sizeof(double), fn[d], sizeof(double), sizeof(double),
                           c->nf, k, s));
  }
  if (mem != VOF_MEM_DEVICE) CK(cudaStreamSynchronize(s));
  return VOF_OK;
}

vof_status vof_get_neighbors(vof_ctx* c, int64_t* ptr, int32_t* idx, int64_t* count) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (count) *count = c->nnb;
  if (ptr) CK(cudaMemcpy(ptr, c->nb_ptr, sizeof(int64_t) * (c->nc + 1), cudaMemcpyDeviceToHost));
  if (idx) CK(cudaMemcpy(idx, c->nb, sizeof(int32_t) * c->nnb, cudaMemcpyDeviceToHost));
  return VOF_OK;
}

vof_status vof_get_candidates(vof_ctx* c, const int32_t* faces, int n, int64_t* out_ptr,
                              int32_t* out_idx, int64_t cap) {
  if (!c || !faces || !out_ptr || n < 0) return fail(VOF_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i)
    if (faces[i] < 0 || faces[i] >= c->nf) return fail(VOF_EINVAL, "face index out of range");
  if (n == 0) { out_ptr[0] = 0; return VOF_OK; }
  const int64_t stride = 128;
  int32_t *df, *dout, *dcnt;
  CK(cudaMalloc(&df, sizeof(int32_t) * n));
  CK(cudaMalloc(&dout, sizeof(int32_t) * n * stride));
  CK(cudaMalloc(&dcnt, sizeof(int32_t) * n));
  CK(cudaMemcpy(df, faces, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  CK(launch_candidates(c, df, n, stride, dout, dcnt, 0));
  std::vector<int32_t> h(n * stride), hc(n);
  CK(cudaMemcpy(h.data(), dout, sizeof(int32_t) * n * stride, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hc.data(), dcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  cudaFree(df); cudaFree(dout); cudaFree(dcnt);
  out_ptr[0] = 0;
  for (int i = 0; i < n; ++i) {
    if (hc[i] > stride) return fail(VOF_ECAPACITY, "more than 128 candidates for a face");
    out_ptr[i + 1] = out_ptr[i] + hc[i];
    if (out_idx) {
      if (out_ptr[i + 1] > cap) return fail(VOF_ECAPACITY, "out_idx too small");
      std::memcpy(out_idx + out_ptr[i], h.data() + i * stride, sizeof(int32_t) * hc[i]);
    }
  }
  return VOF_OK;
}

vof_status vof_get_flux_polyhedra(vof_ctx* c, const vof_velocity* vel, double t, double dt,
                                  const int32_t* faces, int n, double* verts, int32_t* counts) {
  if (!c || !faces || !verts || !counts || n < 0) return fail(VOF_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i)
    if (faces[i] < 0 || faces[i] >= c->nf) return fail(VOF_EINVAL, "face index out of range");
  if (!vel) return fail(VOF_EINVAL, "velocity is NULL");
  std::vector<vof_velocity> vv(c->n_grids, *vel);
  std::vector<double> tt(c->n_grids, t), dd(c->n_grids, dt);
  vof_status st = ensure_velocity(c, vv.data(), 0);
  if (st != VOF_OK) return st;
  st = upload_params(c, tt.data(), dd.data(), 0);
  if (st != VOF_OK) return st;
  if (n == 0) return VOF_OK;
  const int NBV = VOF_MAX_POLY_VERTS;
  int32_t *df, *dcnt;
  double* dv;
  CK(cudaMalloc(&df, sizeof(int32_t) * n));
  CK(cudaMalloc(&dcnt, sizeof(int32_t) * n));
  CK(cudaMalloc(&dv, sizeof(double) * n * NBV * 3));
  CK(cudaMemset(dv, 0, sizeof(double) * n * NBV * 3));
  CK(cudaMemcpy(df, faces, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  CK(launch_polyhedra(c, df, n, dv, dcnt, 0));
  CK(cudaMemcpy(verts, dv, sizeof(double) * n * NBV * 3, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(counts, dcnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  cudaFree(df); cudaFree(dcnt); cudaFree(dv);
  return VOF_OK;
}

vof_status vof_get_stats(vof_ctx* c, vof_stats* out, void* stream) {
  if (!c || !out) return fail(VOF_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_volume_sum(c, s));
  unsigned long long* h = (unsigned long long*)c->pinned;
  double* hd = (double*)((char*)c->pinned + 1024);
  CK(cudaMemcpyAsync(h, c->cnt, sizeof(unsigned long long) * kNCnt, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hd, c->red + kRedSlots - 5, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out->n_interfacial = (int64_t)h[kNIcells];
  out->n_active_faces = (int64_t)h[kNAfaces];
  out->n_truncations = (int64_t)h[kNTrunc];
  out->n_overflow = (int64_t)h[kNOverflow];
  out->n_degenerate = (int64_t)h[kNDegen];
  out->n_edgeon = (int64_t)h[kNEdgeOn];
  out->clip_loss = hd[kAccClip];
  out->boundary_outflow = hd[kAccBoundary];
  out->cutoff_loss = hd[kAccCutoff];
  out->volume = hd[3];
  out->ebound = hd[4];
  out->n_clipped = (int64_t)h[kNClipped];
  out->n_repaired = (int64_t)std::min<unsigned long long>(h[kNRepFaces], (unsigned long long)c->rep_cap);
  out->n_escaped = (int64_t)h[kNEscape];
  if (out->n_escaped > 0)
    return fail(VOF_ECFL, std::to_string(out->n_escaped) +
                              " flux polyhedra of the last advect reached past their candidate "
                              "cells (CFL too large for this grid); the stats are filled in");
  return VOF_OK;
}

}  // extern "C"

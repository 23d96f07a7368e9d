// Shared declarations of the gvof CUDA library: device views of the mesh and
// state, the context, velocity evaluation, and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "../../include/vof.h"

#define GVOF_FULL 0xffffffffu

namespace gvof {

constexpr int kSMs = 152;  // GB300
constexpr int kMaxFaceVerts = 8;
constexpr int kMaxEmfpaVerts = 6;  // 5I+1 EMFPA faces fit the 32-face capacity
constexpr int kMaxLsfirIter = 16;  // LSFIR outer iterations at most
// flux polyhedra built ahead of the flux kernel: vertex slots per face and
// the faces a context keeps room for (later active faces are built in the
// flux kernel itself, with the same arithmetic)
constexpr int kFmSlots = VOF_MAX_POLY_VERTS;
// candidate cells listed per prebuilt polyhedron (FP32 path); a face with
// more is left to the flux kernel's own search
constexpr int kPreCand = 32;
// the lists are built where cells have few node neighbours (hexahedral
// grids: 26); on tetrahedral grids (50 and more) most faces' candidate sets
// exceed the list and the flux kernel's truncations dominate anyway
inline bool cand_lists_on(const vof_options& o, int64_t nnb, int64_t nc) {
  return o.precision == VOF_PREC_MIXED && nnb <= 30 * nc;
}
constexpr int64_t kFmCap = int64_t(4) << 20;
static_assert(3 * kMaxEmfpaVerts + 1 <= VOF_MAX_POLY_VERTS && 2 * kMaxFaceVerts + 1 <= VOF_MAX_POLY_VERTS,
              "polyhedron export stride");

struct Vel {
  int kind;
  double period, omega, cx, cy, cz, ux, uy, uz;
};

// per-grid parameters of one step, in device memory so that the launches of
// a step take no per-step argument (and can be replayed as a CUDA graph)
struct GridParam {
  Vel vel;
  double g;    // time factor of the field at t + dt/2
  double dt;
  double gdt;  // g * dt
  double pad;
};

// grid of face f: faces of grid i are [face_off[i], face_off[i+1])
__device__ __forceinline__ int grid_of(const int64_t* face_off, int n_grids, int64_t f) {
  int lo = 0, hi = n_grids;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (face_off[mid] <= f) lo = mid; else hi = mid;
  }
  return lo;
}

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
  const uint8_t* convex;          // 0: not convex, 1: convex, 2: convex box with axis-aligned faces
  const int64_t* face_off;        // [n_grids + 1] first face of each grid
  int n_grids;
  // mixed-precision copies (allocated for VOF_PREC_MIXED only): absolute
  // positions as (hi, lo) float pairs, hi = fl(x), lo = fl(x - hi), so that
  // differences of nearby points are formed in FP32 without losing the
  // digits an FP32 absolute coordinate would drop; directions in FP32
  const float2 *vx2, *vy2, *vz2;
  const float2 *fcx2, *fcy2, *fcz2;
  const float *fnx32, *fny32, *fnz32, *fa32;
  const float2 *ccx2, *ccy2, *ccz2;
  const float2* bb2;
  const float* cvol32;
  // per cell face entry (cell -> faces CSR order): inward unit normal n and
  // d = n.(p_face - x_cell), so that the cell is n.(x - x_cell) >= d on
  // every face plane (convex cells; FP32, mixed only)
  const float4* cpl32;
  // per node: radius of a ball about the node that its cells cover (0 on
  // the domain boundary); a point that close to the node lies in one of them
  const float* rstar;
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
  float *nx32, *ny32, *nz32, *C32;  // FP32 copies of the planes (mixed only)
  const GridParam* gp;              // [n_grids] parameters of the current step
  // LSFIR (allocated with VOF_RECON_LSFIR only): PLIC vertex-average
  // centres by cell (FP64: absolute; mixed: FP32 offsets from the cell
  // centroid), accepted normals by band position, and per outer iteration
  // the largest accepted turn (bit pattern of a non-negative double)
  double *lxp, *lyp, *lzp;
  float *lxr, *lyr, *lzr;
  double *lnx, *lny, *lnz;
  float *lnx32, *lny32, *lnz32;
  unsigned long long* lturn;
  // prebuilt flux polyhedra of the first fm_cap active faces: vertices
  // [(w kFmSlots + k) 3 + d], frame [w 7] (L, lo xyz, hi
  // xyz), meta [w] (I | degenerate << 8 | edge-on << 16 | built << 24),
  // split [w]; in the precision of the path (float or double)
  void* fm_v;
  void* fm_f;
  uint32_t *fm_meta, *fm_split;
  int64_t fm_cap;
  // FP32 path: the candidate cells of each prebuilt polyhedron [w kPreCand]
  // and their count | any empty << 6 | any full << 7 (count 63: not listed)
  int32_t* fm_cand;
  uint8_t* fm_cinfo;
  // domain bounding box per grid [6 * n_grids] (lo xyz, hi xyz): a flux
  // polyhedron vertex outside it is outside the domain (no fluid there)
  const double* dombox;
  // mixed precision reconciliation: per face, 1 when the last flux kernel's
  // V_F is exact (shortcut or a polyhedron inside one cell's fluid or empty
  // part); F before the update (band cells); risk, adjusted-face and
  // re-update lists
  uint8_t* fexact;
  double* Fprev;
  int32_t *risk, *repf, *repc, *stamp_r;
  double *Eexc, *Sroom;  // per risk cell: excess and neighbours' room
  int64_t rep_cap;
  // coverage bits of each active face's flux polyhedron by active position
  // (k_coverage in k_flux.cu)
  uint8_t* cover8;
};

enum Cnt {
  kNIcells = 0,
  kNAfaces = 1,
  kNTrunc = 2,
  kNOverflow = 3,
  kNDegen = 4,
  kNEdgeOn = 5,
  kUmax = 6,  // 3 slots: max |u0| per axis (bit pattern of non-negative doubles)
  // band-limited sweeps (see k_sweep.cu)
  kNBandCells = 9,   // cells whose F the update may change this step
  kNBandNodes = 10,  // nodes of those cells
  kEpoch = 11,       // step counter for the de-duplication stamps
  kBandCellsOk = 12, // the band cell list of the last advect is valid
  kBandNodesOk = 13, // the band node list of the last reconstruction is valid
  kNInitList = 14,   // cells the initial surface may cross (vof_init_fraction)
  kFluxNext = 15,    // next active face a flux warp takes (reset before each launch)
  kReconNext = 16,   // next interfacial cell a reconstruction warp takes (likewise)
  // mixed precision: reconciliation of the FP32 face-volume noise of cells
  // at the bounds (k_sweep.cu) and the candidate-ring escape count
  kNClipped = 17,    // cells clipped to [0, 1] by the last update
  kNEscape = 18,     // flux polyhedra with a vertex outside every candidate cell
  kNRepFaces = 19,   // faces adjusted this advect (listed once per round)
  kRepLo = 20,       // first adjusted face of the current round
  kNRisk = 21,       // cells appended to the risk list this advect
  kRiskLo = 22,      // risk cells of the current round: [kRiskLo, kRiskHi)
  kRiskHi = 23,
  kNRepCells = 24,   // cells re-updated in the current round
  kNCnt = 25
};
// rounds of the mixed path's reconciliation of FP32 face-volume noise
constexpr int kRepairRounds = 3;
constexpr int kRedSlots = 2 * 1024;
// volume bookkeeping: per-block running sums, one region each (fixed block
// counts, so every sum is formed in the same order every step)
constexpr int kAccSlots = kSMs * 16;
enum Acc { kAccClip = 0, kAccBoundary = 1, kAccCutoff = 2, kNAcc = 3 };

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
  } else if (v.kind == VOF_VEL_DEFORMATION2D) {
    double sx, cx, sz, cz;
    sincospi(x, &sx, &cx);
    sincospi(z, &sz, &cz);
    u = -2.0 * sx * sx * sz * cz;
    w = 0.0;
    s = 2.0 * sz * sz * sx * cx;
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
  } else if (v.kind == VOF_VEL_DEFORMATION2D) {
    float sx, cx, sz, cz;
    sincospif(x, &sx, &cx);
    sincospif(z, &sz, &cz);
    u = -2.0f * sx * sx * sz * cz;
    w = 0.0f;
    s = 2.0f * sz * sz * sx * cx;
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

// absolute coordinates in the two precisions: double, or a (hi, lo) float
// pair whose difference with another pair is formed in FP32 as
// (a.hi - b.hi) + (a.lo - b.lo)
template <typename G>
struct Prec;
template <>
struct Prec<double> {
  using A = double;
};
template <>
struct Prec<float> {
  using A = float2;
};
__device__ __forceinline__ double rel(double a, double b) { return a - b; }
__device__ __forceinline__ float rel(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

// the bounding box of cell k (lo x y z, hi x y z) from GeoView::bb: the FP64
// path keeps six arrays of n_cell; the FP32 path one 48-byte record of (hi,
// lo) pairs per cell, read as three 16-byte loads
template <typename G>
__device__ __forceinline__ void cell_box(const typename Prec<G>::A* bb, int64_t nc, int64_t k,
                                         typename Prec<G>::A* b) {
  if constexpr (sizeof(G) == 4) {
    const float4* q = reinterpret_cast<const float4*>(bb) + 3 * k;
    const float4 u = q[0], v = q[1], w = q[2];
    b[0] = make_float2(u.x, u.y); b[1] = make_float2(u.z, u.w);
    b[2] = make_float2(v.x, v.y); b[3] = make_float2(v.z, v.w);
    b[4] = make_float2(w.x, w.y); b[5] = make_float2(w.z, w.w);
  } else {
    for (int d = 0; d < 6; ++d) b[d] = bb[d * nc + k];
  }
}

// mesh and plane arrays as seen by the band kernels of precision G
template <typename G>
struct GeoView {
  using A = typename Prec<G>::A;
  const A *vx, *vy, *vz;      // vertices
  const A *fcx, *fcy, *fcz;   // face centroids
  const G *fnx, *fny, *fnz;   // face unit normals (out of the owner)
  const G* fa;                // face areas
  const A *ccx, *ccy, *ccz;   // cell centroids
  const A* bb;                // cell bounding boxes [6 * nc] (read with cell_box)
  const G* cvol;              // cell volumes
  const G *pnx, *pny, *pnz, *pC;  // PLIC planes (read)
};

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
  float2 *vx2, *vy2, *vz2, *fcx2, *fcy2, *fcz2, *ccx2, *ccy2, *ccz2;
  float2* bb2;  // [6 n_cell]: lo xyz, hi xyz of cell c at 6 c .. 6 c + 5
  float *fnx32, *fny32, *fnz32, *fa32, *cvol32;
  float4* cpl32;
  float* rstar;
  float *nx32, *ny32, *nz32, *C32;
  // LSFIR scratch (see DevState)
  double *lxp, *lyp, *lzp;
  float *lxr, *lyr, *lzr;
  double *lnx, *lny, *lnz;
  float *lnx32, *lny32, *lnz32;
  unsigned long long* lturn;
  void *fm_v, *fm_f;
  uint32_t *fm_meta, *fm_split;
  int64_t fm_cap;
  int32_t* fm_cand;
  uint8_t* fm_cinfo;
  double* dombox;
  uint8_t* fexact;
  double* Fprev;
  int32_t *risk, *repf, *repc, *stamp_r;
  double *Eexc, *Sroom;  // per risk cell: excess and neighbours' room
  int64_t rep_cap;
  uint8_t* cover8;
  // cell lists of a partitioned grid (vof_halo_lists): entries, offsets
  // (host), and the partial sums of vof_list_volume
  int32_t* lists;
  int64_t n_list_cells;
  std::vector<int64_t>* list_ptr;
  double* list_part;
  // state (device)
  double* F;
  double *nx, *ny, *nz, *C;
  int8_t *tv, *tf, *tc;
  double *Vd, *VF, *srate;
  int32_t *icells, *afaces;
  unsigned long long* cnt;
  double* red;
  double* acc;  // [kNAcc * kAccSlots] volume bookkeeping since the last set_fraction
  int32_t* bfaces;  // boundary faces (no neighbour)
  int64_t nbf;
  // band-limited sweeps: node -> faces CSR, per-entity stamps, band lists
  int64_t* vf_ptr;
  int32_t* vf;
  int32_t *stamp_c, *stamp_v, *stamp_f;
  int32_t *bcells, *bnodes;
  // host-side caches
  bool vel_valid;
  bool recon_valid;
  int max_face_verts;
  int max_cell_faces;
  int max_cell_verts;
  int64_t bytes;
  void* pinned;  // small pinned host buffer for counters / sums
  // batching: grids joined into this context
  int n_grids;
  int64_t* face_off_d;                      // device copy of face offsets
  std::vector<int64_t>* cell_off, *face_off, *vert_off;  // host offsets [n_grids + 1]
  std::vector<double>* hmin_g;              // [3 * n_grids]
  std::vector<double>* umax_g;              // [3 * n_grids]
  std::vector<gvof::Vel>* vel_g;            // cached velocity per grid
  gvof::GridParam* gp_d;                    // [n_grids] device table
  gvof::GridParam* gp_ring;                 // pinned ring [kRing * n_grids]
  cudaEvent_t ring_ev[16];  // one per ring slot
  int ring_pos;
  unsigned long long* umax_d;               // [3 * n_grids]
  // CUDA graph of one step (optional)
  cudaGraph_t graph;
  cudaGraphExec_t graph_exec;
  int graph_step;                           // 1: advect + reconstruct, 0: advect only
  // launch shapes (autotuned)
  int flux_blocks, recon_blocks;
  int faces_per_warp;   // 1 or 2: lane-group width 32 or 16 of the flux kernel
  bool half_ok;         // the grid allows faces_per_warp = 2
  int64_t fm_use;       // faces whose polyhedra are prebuilt (0 or fm_cap)
  // optional per-phase timing (events recorded around each launch)
  bool timing;
  int n_ev_pairs;
  cudaEvent_t ev[2 * 256];
  int ev_phase[256];
  int ev_n[256];
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
  m.convex = c->convex;
  m.face_off = c->face_off_d;
  m.n_grids = c->n_grids;
  m.vx2 = c->vx2; m.vy2 = c->vy2; m.vz2 = c->vz2;
  m.fcx2 = c->fcx2; m.fcy2 = c->fcy2; m.fcz2 = c->fcz2;
  m.fnx32 = c->fnx32; m.fny32 = c->fny32; m.fnz32 = c->fnz32; m.fa32 = c->fa32;
  m.ccx2 = c->ccx2; m.ccy2 = c->ccy2; m.ccz2 = c->ccz2; m.bb2 = c->bb2; m.cvol32 = c->cvol32;
  m.cpl32 = c->cpl32;
  m.rstar = c->rstar;
  return m;
}

inline DevState state_view(const vof_ctx* c) {
  DevState s;
  s.F = c->F; s.nx = c->nx; s.ny = c->ny; s.nz = c->nz; s.C = c->C;
  s.tv = c->tv; s.tf = c->tf; s.tc = c->tc; s.Vd = c->Vd; s.VF = c->VF; s.srate = c->srate;
  s.icells = c->icells; s.afaces = c->afaces; s.cnt = c->cnt; s.red = c->red;
  s.nx32 = c->nx32; s.ny32 = c->ny32; s.nz32 = c->nz32; s.C32 = c->C32;
  s.gp = c->gp_d;
  s.lxp = c->lxp; s.lyp = c->lyp; s.lzp = c->lzp;
  s.lxr = c->lxr; s.lyr = c->lyr; s.lzr = c->lzr;
  s.lnx = c->lnx; s.lny = c->lny; s.lnz = c->lnz;
  s.lnx32 = c->lnx32; s.lny32 = c->lny32; s.lnz32 = c->lnz32;
  s.lturn = c->lturn;
  s.fm_v = c->fm_v; s.fm_f = c->fm_f; s.fm_meta = c->fm_meta; s.fm_split = c->fm_split;
  s.fm_cand = c->fm_cand; s.fm_cinfo = c->fm_cinfo;
  s.fm_cap = c->fm_use;
  s.dombox = c->dombox;
  s.fexact = c->fexact; s.Fprev = c->Fprev;
  s.risk = c->risk; s.repf = c->repf; s.repc = c->repc; s.stamp_r = c->stamp_r;
  s.Eexc = c->Eexc; s.Sroom = c->Sroom;
  s.rep_cap = c->rep_cap;
  s.cover8 = c->cover8;
  return s;
}

template <typename G>
GeoView<G> geo_view(const vof_ctx* c);

template <>
inline GeoView<double> geo_view<double>(const vof_ctx* c) {
  GeoView<double> g;
  g.vx = c->x; g.vy = c->y; g.vz = c->z;
  g.fcx = c->fcx; g.fcy = c->fcy; g.fcz = c->fcz;
  g.fnx = c->fnx; g.fny = c->fny; g.fnz = c->fnz; g.fa = c->fa;
  g.ccx = c->ccx; g.ccy = c->ccy; g.ccz = c->ccz; g.bb = c->bb; g.cvol = c->cvol;
  g.pnx = c->nx; g.pny = c->ny; g.pnz = c->nz; g.pC = c->C;
  return g;
}

template <>
inline GeoView<float> geo_view<float>(const vof_ctx* c) {
  GeoView<float> g;
  g.vx = c->vx2; g.vy = c->vy2; g.vz = c->vz2;
  g.fcx = c->fcx2; g.fcy = c->fcy2; g.fcz = c->fcz2;
  g.fnx = c->fnx32; g.fny = c->fny32; g.fnz = c->fnz32; g.fa = c->fa32;
  g.ccx = c->ccx2; g.ccy = c->ccy2; g.ccz = c->ccz2; g.bb = c->bb2; g.cvol = c->cvol32;
  g.pnx = c->nx32; g.pny = c->ny32; g.pnz = c->nz32; g.pC = c->C32;
  return g;
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
  if (v.kind == VOF_VEL_DEFORMATION || v.kind == VOF_VEL_DEFORMATION2D)
    return std::cos(3.14159265358979323846 * t / v.period);
  return 1.0;
}

// message returned by vof_last_error() on this thread
void set_last_error(const char* msg);

// ------------------------------------------------------------ launchers
// set-up (k_setup.cu)
cudaError_t launch_face_geometry(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_cell_geometry(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_node_star(const vof_ctx* c, cudaStream_t s);  // rstar
cudaError_t launch_velocity_setup(const vof_ctx* c, cudaStream_t s);  // velocities in gp_d
cudaError_t launch_mixed_copies(const vof_ctx* c, cudaStream_t s);
// sweeps (k_sweep.cu)
cudaError_t launch_cell_tags(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_node_tags(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_face_sweep(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_update(const vof_ctx* c, cudaStream_t s);
// mixed precision: reconciliation of the FP32 face-volume noise of cells the
// clip would cut and the re-update of their cells (kRepairRounds rounds),
// then the final clip and the boundary outflow
cudaError_t launch_repair(const vof_ctx* c, cudaStream_t s);
int repair_launch_count();
// F from Fin (device); keeps the band-limited sweeps when only band cells change
cudaError_t launch_set_fraction(const vof_ctx* c, const double* Fin, cudaStream_t s);
cudaError_t launch_face_flux_export(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_volume_sum(const vof_ctx* c, cudaStream_t s);  // writes red[0], red[1]
// initial volume fraction (k_init.cu)
cudaError_t launch_init_fraction(const vof_ctx* c, const vof_shape* shape, int ndiv, cudaStream_t s);
// reconstruction (k_recon.cu)
// LSGIR (+ the LSFIR outer iteration when the context asks for it)
cudaError_t launch_reconstruct(const vof_ctx* c, cudaStream_t s);
int reconstruct_launch_count(const vof_ctx* c);
// flux (k_flux.cu)
// the flux polyhedra of the active faces (up to fm_cap), then the truncations
cudaError_t launch_prebuild(const vof_ctx* c, cudaStream_t s);  // + candidate lists (FP32)
bool prebuild_lists(const vof_ctx* c);  // launch_prebuild also builds the candidate lists
struct HostConn;
// vof_batch_create with each grid's connectivity already built (the server
// builds it once, to size the request, and hands it on)
vof_status batch_create_with_conn(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                                  void* stream, vof_ctx** out, const HostConn* const* conns);
cudaError_t launch_flux(const vof_ctx* c, cudaStream_t s);
cudaError_t launch_candidates(const vof_ctx* c, const int32_t* faces, int n, int64_t cap_per_face,
                              int32_t* out, int32_t* counts, cudaStream_t s);
cudaError_t launch_polyhedra(const vof_ctx* c, const int32_t* faces, int n, double* verts,
                             int32_t* counts, cudaStream_t s);

}  // namespace gvof

// Sweeps of one step: tags (Sec. 3.3), the face sweep that finds the faces
// with geometric fluxes, and the cell update of Eq. fnext with the final clip
// (Sec. 2.2). One thread per cell / node / face, coalesced SoA loads,
// warp-aggregated compaction of the work lists.
//
// Band-limited sweeps. The paper's sweeps visit every cell, node and face;
// on a large grid almost all of them are uniform (F = 0 or 1) and stay so.
// A cell's F can change in a step only if one of its faces carries a
// geometric flux (tag 0) or it is interfacial: a cell whose faces all carry
// shortcut fluxes keeps F = 0 exactly, and F = 1 up to the last bit that the
// cut-off restores. So after the first, full, sweeps:
//  - the update visits the band cells: owner and neighbour of every active
//    face, and the interfacial cells (de-duplicated by per-step stamps);
//  - the cut-off and cell tags visit the band cells (every interfacial cell
//    is one of them);
//  - node tags visit the band nodes, the nodes of the band cells (no other
//    node has a cell whose F changed);
//  - the next face sweep visits the faces of the band nodes: a face whose
//    tag changes has a band node, and every face active in the last step
//    lies on a band cell.
// F and every tag are those of the full sweeps. Device flags (counter slots
// kBandCellsOk, kBandNodesOk) select band or full work inside the kernels,
// so a captured CUDA graph stays valid for every replay.
#include <cstring>

#include "vof_common.cuh"

namespace gvof {
namespace {

inline int grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  int64_t cap = (int64_t)kSMs * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// append `item` to list when `pred` holds; one atomic per warp
__device__ __forceinline__ void warp_append(bool pred, int32_t item, int32_t* list,
                                            unsigned long long* counter) {
  unsigned m = __ballot_sync(GVOF_FULL, pred);
  if (m == 0) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(GVOF_FULL, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1))] = item;
}

// FP64 comparisons run on the (narrow) FP64 pipe of the GPU; the sweeps
// compare the bit patterns instead: for doubles, x < y <=> bits(x) < bits(y)
// whenever y > 0 (negative x have negative bit patterns as int64)
constexpr long long kOneBits = 0x3FF0000000000000LL;
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) << 1) == 0; }

// sum over the block in a fixed order (valid in thread 0); every thread of the
// block must call it
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sb[32];
  __syncthreads();
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GVOF_FULL, v, o);
  if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sb[i];
  return t;
}
__device__ __forceinline__ bool is_one(double x) { return dbits(x) == kOneBits; }

// de-duplicating claim of an entity for this step's list
__device__ __forceinline__ bool claim(int32_t* stamp, int64_t i, int32_t epoch) {
  return atomicExch(stamp + i, epoch) != epoch;
}

// cut-off of uniform cells and cell tags (Sec. 2.1, Sec. 3.3); interfacial
// cells are appended to their list. Visits all cells, or the band cells when
// the last update produced them.
__global__ void k_cell_tags(int64_t nc, long long eps_bits, long long ome_bits, double* F,
                            const double* cvol, int8_t* tc, int32_t* icells,
                            unsigned long long* cnt, double* acc_cut, const int32_t* bcells) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double cut = 0.0;  // volume the cut-off removes (Sec. 2.1)
  const bool band = cnt[kBandCellsOk] != 0;
  const int64_t n = band ? (int64_t)cnt[kNBandCells] : nc;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    const bool in = i < n;
    const int64_t c = in ? (band ? bcells[i] : i) : 0;
    int8_t t = -1;
    if (in) {
      const double f = F[c];
      const long long b = dbits(f);
      if (b < eps_bits) {  // F < eps
        t = -1;
        if (b != 0) { F[c] = 0.0; cut += cvol[c] * f; }
      } else if (b > ome_bits) {  // F > 1 - eps
        t = 1;
        if (b != kOneBits) { F[c] = 1.0; cut += cvol[c] * (f - 1.0); }
      } else {
        t = 0;
      }
      tc[c] = t;
    }
    warp_append(in && t == 0, (int32_t)c, icells, cnt + kNIcells);
  }
  const double s = block_sum(cut);
  if (threadIdx.x == 0) acc_cut[blockIdx.x] += s;
}

// node value F* by inverse-distance weighting of the cells sharing the node
// and node tags (Sec. 3.3). Nodes whose cells are all empty or all full take
// F* = 0 or 1 exactly without forming the weights.
template <typename G>
__global__ void k_node_tags(DevMesh M, const double* F, double eps, int8_t* tv,
                            const unsigned long long* cnt, const int32_t* bnodes) {
  const bool band = cnt[kBandCellsOk] != 0;
  const int64_t n = band ? (int64_t)cnt[kNBandNodes] : M.nv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = band ? bnodes[i] : i;
    int64_t q0 = M.vc_ptr[v], q1 = M.vc_ptr[v + 1];
    bool allz = true, allo = true;
    for (int64_t q = q0; q < q1; ++q) {
      const double f = F[M.vc[q]];
      allz &= is_zero(f);
      allo &= is_one(f);
    }
    int8_t t;
    if (allz) t = -1;
    else if (allo) t = 1;
    else {
      double xv = M.x[v], yv = M.y[v], zv = M.z[v];
      double num = 0.0, den = 0.0;
      for (int64_t q = q0; q < q1; ++q) {
        int c = M.vc[q];
        G dx = (G)(xv - M.ccx[c]), dy = (G)(yv - M.ccy[c]), dz = (G)(zv - M.ccz[c]);
        G r2 = dx * dx + dy * dy + dz * dz;
        double w = (double)(G(1) / sqrt(r2));
        num += w * F[c];
        den += w;
      }
      double fs = num / den;
      t = fs < eps ? -1 : (fs > 1.0 - eps ? 1 : 0);
    }
    tv[v] = t;
  }
}

// a list whose items each own a short CSR range (the faces of a node, the
// nodes of a cell), taken by sub-warps of S lanes: 32 / S items per warp at
// once, each sub-warp's lanes striding over its item's range. The warp's
// loops keep a uniform trip count (the longest range among its items), so
// warp-wide ballots (warp_append) see the whole warp.
template <int S>
struct SubWarp {
  static_assert(32 % S == 0, "S divides the warp");
  const int sub, sl;
  __device__ SubWarp() : sub((threadIdx.x & 31) / S), sl(threadIdx.x % S) {}
  // the warp's first item and the stride over the list
  __device__ int64_t first() const {
    return ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * (32 / S);
  }
  __device__ int64_t stride() const { return (((int64_t)gridDim.x * blockDim.x) >> 5) * (32 / S); }
  // the longest of the warp's ranges
  __device__ int64_t max_len(int64_t len) const {
    for (int o = S; o < 32; o <<= 1) {
      const int64_t x = __shfl_xor_sync(GVOF_FULL, len, o);
      len = x > len ? x : len;
    }
    return len;
  }
};
// lanes per band node in the face sweep (a hex grid's node has 12 faces)
// and per band cell in the node list (a hex has 8 nodes)
constexpr int kSweepLanes = 16;
constexpr int kNodeLanes = 8;

// face sweep: face tags from node tags, V_d = g(t+dt/2) (u0.n) A dt,
// V_F = 0 on tag -1 faces, V_F = V_d on tag 1 faces (no geometry, Sec. 3.3);
// tag 0 faces are appended to the active list for the flux kernel
__device__ __forceinline__ int8_t face_tag(const DevMesh& M, const int8_t* tv, int64_t f) {
  const int64_t b = M.fptr[f], e = M.fptr[f + 1];
  bool allm = true, allp = true;
  for (int64_t k = b; k < e; ++k) {
    const int8_t x = tv[M.fvert[k]];
    allm &= (x == -1);
    allp &= (x == 1);
  }
  return allm ? -1 : (allp ? 1 : 0);
}

// start of a step: new stamp epoch, empty band cell list
__global__ void k_band_begin(unsigned long long* cnt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cnt[kEpoch] += 1;
    cnt[kNBandCells] = 0;
  }
}

// face tags and the active list: all faces, or (band nodes valid) one
// sub-warp per band node over the faces that contain it
__global__ void k_face_sweep(DevMesh M, const int8_t* tv, int8_t* tf, int32_t* afaces,
                             unsigned long long* cnt, const int64_t* vf_ptr, const int32_t* vf,
                             const int32_t* bnodes, int32_t* stamp_f) {
  if (cnt[kBandNodesOk] == 0) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < M.nf; base += stride) {
      int64_t f = base + threadIdx.x;
      bool in = f < M.nf;
      int8_t t = 0;
      if (in) {
        t = face_tag(M, tv, f);
        tf[f] = t;
      }
      warp_append(in && t == 0, (int32_t)f, afaces, cnt + kNAfaces);
    }
    return;
  }
  const int32_t epoch = (int32_t)cnt[kEpoch];
  const int64_t nb = (int64_t)cnt[kNBandNodes];
  SubWarp<kSweepLanes> sw;
  for (int64_t i0 = sw.first(); i0 < nb; i0 += sw.stride()) {
    const int64_t i = i0 + sw.sub;
    int64_t q0 = 0, q1 = 0;
    if (i < nb) {
      const int v = bnodes[i];
      q0 = vf_ptr[v];
      q1 = vf_ptr[v + 1];
    }
    const int64_t len = q1 - q0, rounds = sw.max_len(len);
    for (int64_t k = sw.sl; k - sw.sl < rounds; k += kSweepLanes) {
      bool act = false;
      int f = 0;
      if (k < len) {
        f = vf[q0 + k];
        const int8_t t = face_tag(M, tv, f);
        tf[f] = t;  // every sub-warp that meets f writes the same tag
        act = t == 0 && claim(stamp_f, f, epoch);
      }
      warp_append(act, f, afaces, cnt + kNAfaces);
    }
  }
}

// band cells: owner and neighbour of each active face, and the interfacial
// cells, each once
__global__ void k_band_cells(DevMesh M, const int32_t* afaces, const int32_t* icells,
                             unsigned long long* cnt, int32_t* stamp_c, int32_t* bcells) {
  const int32_t epoch = (int32_t)cnt[kEpoch];
  const int64_t na = (int64_t)cnt[kNAfaces], ni = (int64_t)cnt[kNIcells];
  const int64_t n = na + ni;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    int c0 = -1, c1 = -1;
    if (i < na) {
      const int f = afaces[i];
      c0 = M.own[f];
      c1 = M.nbr[f];
    } else if (i < n) {
      c0 = icells[i - na];
    }
    const bool p0 = c0 >= 0 && claim(stamp_c, c0, epoch);
    warp_append(p0, c0, bcells, cnt + kNBandCells);
    const bool p1 = c1 >= 0 && claim(stamp_c, c1, epoch);
    warp_append(p1, c1, bcells, cnt + kNBandCells);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) cnt[kBandCellsOk] = 1;
}

// band nodes: the nodes of the band cells, each once (one sub-warp per cell)
__global__ void k_band_nodes(DevMesh M, const int32_t* bcells, unsigned long long* cnt,
                             int32_t* stamp_v, int32_t* bnodes) {
  if (cnt[kBandCellsOk] == 0) return;
  const int32_t epoch = (int32_t)cnt[kEpoch];
  const int64_t n = (int64_t)cnt[kNBandCells];
  SubWarp<kNodeLanes> sw;
  for (int64_t i0 = sw.first(); i0 < n; i0 += sw.stride()) {
    const int64_t i = i0 + sw.sub;
    int64_t q0 = 0, q1 = 0;
    if (i < n) {
      const int c = bcells[i];
      q0 = M.cv_ptr[c];
      q1 = M.cv_ptr[c + 1];
    }
    const int64_t len = q1 - q0, rounds = sw.max_len(len);
    for (int64_t k = sw.sl; k - sw.sl < rounds; k += kNodeLanes) {
      int v = 0;
      bool p = false;
      if (k < len) {
        v = M.cv[q0 + k];
        p = claim(stamp_v, v, epoch);
      }
      warp_append(p, v, bnodes, cnt + kNBandNodes);
    }
  }
}

// vof_set_fraction: F from Fin. The band-limited sweeps stay valid when every
// cell whose value changes is a band cell of the last advect (the cells the
// next sweeps revisit anyway: the argument above holds for any change of
// their F); a change anywhere else, or with no band current, makes the next
// sweeps full. Flags only go from valid to invalid, so blocks that read them
// before or after another block clears them reach the same end state.
__global__ void k_set_fraction(int64_t nc, const double* Fin, double* F, const int32_t* stamp_c,
                               unsigned long long* cnt) {
  const bool band = cnt[kBandCellsOk] != 0;
  const int32_t epoch = (int32_t)cnt[kEpoch];
  int outside = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double f = Fin[i];
    if (dbits(f) != dbits(F[i])) {
      F[i] = f;
      outside |= (!band || stamp_c[i] != epoch) ? 1 : 0;
    }
  }
  if (__syncthreads_or(outside) && threadIdx.x == 0) {
    cnt[kBandCellsOk] = 0;
    cnt[kBandNodesOk] = 0;
  }
}

// end of a reconstruction: the band node list is valid for the next face
// sweep only if this reconstruction was band-limited
__global__ void k_band_end(unsigned long long* cnt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cnt[kBandNodesOk] = cnt[kBandCellsOk];
    cnt[kBandCellsOk] = 0;
  }
}

// Eq. fnext and the clip of Sec. 2.2; red[] receives per-block partial
// E_bound maxima (before the clip)
// V_F of face f: the shortcut of its tag (Sec. 3.3: 0 for tag -1, V_d for
// tag 1), else the flux kernel's value
__device__ __forceinline__ double face_vf(int8_t t, double vd, const double* VF, int f) {
  return t == 0 ? VF[f] : (t == 1 ? vd : 0.0);
}

__device__ __forceinline__ double grid_gdt(const DevMesh& M, const GridParam* gp, int f) {
  return M.n_grids == 1 ? gp[0].gdt : gp[grid_of(M.face_off, M.n_grids, f)].gdt;
}

// V_d = (u0.n) A g dt of each face and V_F from the face tags, written in
// place of the flux kernel's per-face array (read-back of the face volumes)
__global__ void k_face_flux_export(DevMesh M, const int8_t* tf, const double* srate,
                                   const GridParam* gp, double* Vd, double* VF) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < M.nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const double vd = srate[f] * grid_gdt(M, gp, (int)f);
    Vd[f] = vd;
    const int8_t t = tf[f];
    if (t != 0) VF[f] = t == 1 ? vd : 0.0;
  }
}

__device__ __forceinline__ double wsum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GVOF_FULL, v, o);
  return v;
}
__device__ __forceinline__ double srate_vd(const double* srate, int f, double gdt) {
  return srate[f] * gdt;
}

// the time step factor g dt of the grid of cell c (the faces of a cell
// belong to its grid)
__device__ __forceinline__ double cell_gdt(const DevMesh& M, const GridParam* gp, int64_t q0,
                                           int64_t q1) {
  if (M.n_grids > 1 && q1 > q0) {
    const int fs0 = M.cf[q0];
    return gp[grid_of(M.face_off, M.n_grids, fs0 >= 0 ? fs0 : ~fs0)].gdt;
  }
  return gp[0].gdt;
}

// Eq. fnext for cell c from F0 and the face volumes of its faces (V_d formed
// from the face's rate and the grid's g dt, V_F from its tag); n_inexact
// counts the tag-0 faces whose V_F is not exact (mixed path: fexact != NULL)
__device__ __forceinline__ double cell_fnext(const DevMesh& M, const int8_t* tf, const double* srate,
                                             double gdt, const double* VF, const uint8_t* fexact,
                                             int64_t q0, int64_t q1, double F0, double V,
                                             int* n_inexact) {
  double vdt = 0.0, vft = 0.0;
  int ni = 0;
  for (int64_t q = q0; q < q1; ++q) {
    const int fs = M.cf[q];
    const int f = fs >= 0 ? fs : ~fs;
    const double vd = srate[f] * gdt;
    const int8_t t = tf[f];
    const double vf = face_vf(t, vd, VF, f);
    if (fexact && t == 0 && !fexact[f]) ++ni;
    if (fs >= 0) { vdt += vd; vft += vf; }
    else { vdt -= vd; vft -= vf; }
  }
  *n_inexact = ni;
  const double h = vdt / (2.0 * V);
  return (F0 * (1.0 + h) - vft / V) / (1.0 - h);
}

// the mixed path defers the clip of a cell whose Eq. fnext value leaves
// [0, 1] by more than FP64 rounding while some of its face volumes carry
// FP32 error: the reconciliation of that noise comes first (launch_repair)
constexpr double kRiskTol = 1e-14;
static_assert(kRepairRounds >= 1 && kRepairRounds <= 6, "stamp marks epoch * 16 + 2 round (+1)");
__device__ __forceinline__ bool at_risk(double fn, int n_inexact) {
  return n_inexact > 0 && (fn < -kRiskTol || fn > 1.0 + kRiskTol);
}

// append with a capacity: returns false (and appends nothing) past cap
__device__ __forceinline__ bool warp_append_cap(bool pred, int32_t item, int32_t* list,
                                                unsigned long long* counter, int64_t cap) {
  const unsigned m = __ballot_sync(GVOF_FULL, pred);
  if (m == 0) return false;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(GVOF_FULL, base, leader);
  const int64_t pos = (int64_t)base + __popc(m & ((1u << lane) - 1));
  if (pred && pos < cap) { list[pos] = item; return true; }
  return false;
}

// per-block maximum of E_bound into red[kRedSlots / 2 + block] (fmax with
// what an earlier kernel of this advect left there when `merge`)
__device__ __forceinline__ void block_ebound(double eb, double* red, bool merge) {
  for (int o = 16; o > 0; o >>= 1) eb = fmax(eb, __shfl_xor_sync(GVOF_FULL, eb, o));
  __shared__ double s[32];
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s[w] = eb;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, s[i]);
    double* slot = red + kRedSlots / 2 + blockIdx.x;
    *slot = merge ? fmax(*slot, m) : m;
  }
}

// Eq. fnext per band cell and the clip of Sec. 2.2. Mixed path: F before
// the update is kept (Fprev) and a cell at risk (at_risk) is written
// unclipped and listed for the reconciliation instead of being clipped; the
// boundary outflow is then summed after the repair (k_repair_finish).
__global__ void k_update(DevMesh M, DevState S, const int32_t* bfaces, int64_t nbf, double* acc,
                         const int32_t* bcells, int64_t risk_cap, bool mixed) {
  double eb = 0.0;
  double clip = 0.0;  // volume the clip to [0, 1] removes
  double bnd = 0.0;   // fluid that leaves through the domain boundary
  unsigned long long nclip = 0;
  const int64_t n = (int64_t)S.cnt[kNBandCells];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool risky = false;
    int64_t c = 0;
    double fn = 0.0;
    if (i < n) {
      c = bcells[i];
      const int64_t q0 = M.cf_ptr[c], q1 = M.cf_ptr[c + 1];
      const double F0 = S.F[c];
      if (mixed) S.Fprev[c] = F0;
      const double gdt = cell_gdt(M, S.gp, q0, q1);
      // an empty cell that no fluid enters stays exactly empty: Eq. fnext
      // gives 0 for F = 0 and V_FT = 0 whatever V_dT (no FP64 work needed)
      bool skip = false;
      if (is_zero(F0)) {
        bool none = true;
        for (int64_t q = q0; q < q1 && none; ++q) {
          const int fs = M.cf[q];
          const int f = fs >= 0 ? fs : ~fs;
          const int8_t t = S.tf[f];
          none = t == -1 || is_zero(t == 0 ? S.VF[f] : S.srate[f] * gdt);
        }
        skip = none;
      }
      if (!skip) {
        const double V = M.cvol[c];
        int ni = 0;
        fn = cell_fnext(M, S.tf, S.srate, gdt, S.VF, mixed ? S.fexact : nullptr, q0, q1, F0, V, &ni);
        risky = mixed && at_risk(fn, ni);
        if (!risky) {
          eb = fmax(eb, fmax(-V * fn, V * (fn - 1.0)));
          const double fc = fmax(fmin(fn, 1.0), 0.0);
          clip += V * (fn - fc);
          nclip += fc != fn;
          S.F[c] = fc;
        }
      }
    }
    // cells at risk wait for the repair unclipped; past the list's capacity
    // they are clipped here
    if (mixed) {
      const bool listed = warp_append_cap(risky, (int32_t)c, S.risk, S.cnt + kNRisk, risk_cap);
      if (risky) {
        const double V = M.cvol[c];
        if (listed) {
          S.F[c] = fn;
        } else {
          eb = fmax(eb, fmax(-V * fn, V * (fn - 1.0)));
          const double fc = fmax(fmin(fn, 1.0), 0.0);
          clip += V * (fn - fc);
          nclip += fc != fn;
          S.F[c] = fc;
        }
      }
    }
  }
  // boundary faces (owner side only), each once
  if (!mixed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbf; i += stride) {
      const int f = bfaces[i];
      const int8_t t = S.tf[f];
      if (t == -1) continue;
      const double vd = S.srate[f] * grid_gdt(M, S.gp, f);
      bnd += face_vf(t, vd, S.VF, f);
    }
  }
  {
    const double s1 = block_sum(clip);
    if (threadIdx.x == 0) acc[kAccClip * kAccSlots + blockIdx.x] += s1;
    const double s2 = block_sum(bnd);
    if (threadIdx.x == 0) acc[kAccBoundary * kAccSlots + blockIdx.x] += s2;
  }
  for (int o = 16; o > 0; o >>= 1) nclip += __shfl_xor_sync(GVOF_FULL, nclip, o);
  if ((threadIdx.x & 31) == 0 && nclip) atomicAdd(S.cnt + kNClipped, nclip);
  block_ebound(eb, S.red, false);
}

// ---- Mixed precision: FP32 noise reconciliation (Sec. 2.2 with the clip)
// A cell whose Eq. fnext value leaves [0, 1] loses V (F_unclipped - F) to
// the clip. In the FP64 path that loss is rounding (E_bound of Sec. 4.2
// around 1e-22 here). The mixed path's face volumes carry FP32 noise of
// about 1e-7 of a polyhedron (plane offsets and cut points formed in FP32),
// which pushes nearly full or empty cells past the bounds; the clip would
// turn that noise into lost volume. Instead, a cell whose excess is within
// the noise bound of its inexact faces (kNoise times the sum of A^(3/2)
// over them: each flux is formed in face-local FP32 units of sqrt(A), so its
// rounding is a few ulps of A^(3/2) whatever V_d) hands it back
// through those faces to the neighbours that have room (space for an
// overfull cell, fluid for an overdrawn one), in proportion to that room:
// each adjustment changes one face volume, applied with opposite signs to
// its two cells, so the update stays conservative, and no face moves more
// than the noise. Each round re-applies Eq. fnext (from the F before the
// update) to the cells of the adjusted faces; a cell still out of bounds
// goes to the next round, and the last round clips every cell (the paper's
// clip, which then removes rounding only).
constexpr double kNoise = 2e-6;
// and at most this much of the cell's own volume: an overshoot the FP64
// method makes itself (jittered tetrahedra) is left to the clip above it,
// and below it the volume moved stays under the mixed path's F tolerance
constexpr double kNoiseF = 5e-7;

__device__ __forceinline__ int32_t risk_mark(int32_t epoch, int round) { return epoch * 16 + 2 * round; }
__device__ __forceinline__ int32_t upd_mark(int32_t epoch, int round) { return epoch * 16 + 2 * round + 1; }

// start of a round: the risk cells listed since the last round, an empty
// re-update list, the first adjusted face of the round
__global__ void k_repair_begin(unsigned long long* cnt, int64_t risk_cap, int64_t rep_cap) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cnt[kRiskLo] = cnt[kRiskHi];
    cnt[kRiskHi] = cnt[kNRisk] < (unsigned long long)risk_cap ? cnt[kNRisk] : risk_cap;
    cnt[kRepLo] = cnt[kNRepFaces] < (unsigned long long)rep_cap ? cnt[kNRepFaces] : rep_cap;
    cnt[kNRepCells] = 0;
  }
}

// room of cell n for an excess of sign e: space (e > 0) or fluid (e < 0)
__device__ __forceinline__ double room(const DevMesh& M, const double* F, int n, double e) {
  const double f = F[n];
  return M.cvol[n] * (e > 0.0 ? fmax(0.0, 1.0 - f) : fmax(0.0, f));
}

// the risk cells of this round (one warp each, one lane per face): the
// excess E (scaled by 1 - h of Eq. fnext so that moving E out of the cell's
// face sums removes it), the room S of the neighbours across its inexact
// faces, and those faces listed once per round
__global__ void k_risk_cells(DevMesh M, DevState S, int32_t* stamp_f, double* Eexc, double* Sroom,
                             int round) {
  const int32_t epoch = (int32_t)S.cnt[kEpoch];
  const int64_t lo = (int64_t)S.cnt[kRiskLo], hi = (int64_t)S.cnt[kRiskHi];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = lo + w0; i < hi; i += nw) {
    const int c = S.risk[i];
    int mine = 0;
    if (lane == 0) mine = claim(S.stamp_r, c, risk_mark(epoch, round)) ? 1 : 0;
    if (!__shfl_sync(GVOF_FULL, mine, 0)) continue;  // listed twice in this round
    const int64_t q0 = M.cf_ptr[c], q1 = M.cf_ptr[c + 1];
    const double gdt = cell_gdt(M, S.gp, q0, q1);
    double vdt = 0.0, vft = 0.0, vdi = 0.0;
    bool inexact = false;
    int f = 0, other = -1;
    if (q0 + lane < q1) {
      const int fs = M.cf[q0 + lane];
      f = fs >= 0 ? fs : ~fs;
      const double vd = srate_vd(S.srate, f, gdt);
      const int8_t t = S.tf[f];
      const double vf = face_vf(t, vd, S.VF, f);
      vdt = fs >= 0 ? vd : -vd;
      vft = fs >= 0 ? vf : -vf;
      inexact = t == 0 && !S.fexact[f];
      if (inexact) {
        const double a = M.fa[f];
        vdi = a * sqrt(a);
        other = fs >= 0 ? M.nbr[f] : M.own[f];
      }
    }
    vdt = wsum_d(vdt); vft = wsum_d(vft); vdi = wsum_d(vdi);
    const double V = M.cvol[c];
    const double h = vdt / (2.0 * V);
    const double fn = (S.Fprev[c] * (1.0 + h) - vft / V) / (1.0 - h);
    const double ex = V * (fn - fmax(fmin(fn, 1.0), 0.0));
    // an excess beyond the FP32 noise of the inexact faces is not noise (a
    // genuine overshoot of the method, as on jittered tetrahedra): the clip
    // takes it, as in the FP64 path
    const double E = (fabs(ex) <= kNoise * vdi && fabs(ex) <= kNoiseF * V) ? ex * (1.0 - h) : 0.0;
    const double r = (inexact && other >= 0 && E != 0.0) ? room(M, S.F, other, E) : 0.0;
    const double Sr = wsum_d(r);
    if (lane == 0) { Eexc[c] = E; Sroom[c] = Sr; }
    const bool p = r > 0.0 && claim(stamp_f, f, -risk_mark(epoch, round));
    warp_append_cap(p, f, S.repf, S.cnt + kNRepFaces, S.rep_cap);
  }
}

// the adjusted face volumes of this round, one thread per listed face: each
// risk cell on either side moves its share of E, in proportion to the other
// side's room (at most all of its room: E is split over max(S, |E|))
__global__ void k_adjust_faces(DevMesh M, DevState S, const double* Eexc, const double* Sroom,
                               int round) {
  const int32_t mark = risk_mark((int32_t)S.cnt[kEpoch], round);
  const int64_t lo = (int64_t)S.cnt[kRepLo];
  const int64_t hi = min((int64_t)S.cnt[kNRepFaces], S.rep_cap);
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = S.repf[i];
    const int o = M.own[f], n = M.nbr[f];
    double d = 0.0;
    if (S.stamp_r[o] == mark && Eexc[o] != 0.0) {
      const double E = Eexc[o];
      d += E * room(M, S.F, n, E) / fmax(Sroom[o], fabs(E));
    }
    if (S.stamp_r[n] == mark && Eexc[n] != 0.0) {
      const double E = Eexc[n];
      d -= E * room(M, S.F, o, E) / fmax(Sroom[n], fabs(E));
    }
    S.VF[f] += d;  // positive: out of the owner (into the neighbour)
  }
}

// the cells of this round's adjusted faces, each once per round
__global__ void k_repair_cells(DevMesh M, DevState S, int round) {
  const int32_t mark = upd_mark((int32_t)S.cnt[kEpoch], round);
  const int64_t lo = (int64_t)S.cnt[kRepLo];
  const int64_t hi = min((int64_t)S.cnt[kNRepFaces], S.rep_cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = lo + blockIdx.x * (int64_t)blockDim.x; base < hi; base += stride) {
    const int64_t i = base + threadIdx.x;
    int c0 = -1, c1 = -1;
    if (i < hi) {
      const int f = S.repf[i];
      c0 = M.own[f];
      c1 = M.nbr[f];
    }
    const bool p0 = c0 >= 0 && claim(S.stamp_r, c0, mark);
    warp_append_cap(p0, c0, S.repc, S.cnt + kNRepCells, 2 * S.rep_cap);
    const bool p1 = c1 >= 0 && claim(S.stamp_r, c1, mark);
    warp_append_cap(p1, c1, S.repc, S.cnt + kNRepCells, 2 * S.rep_cap);
  }
}

// Eq. fnext again for the cells of the adjusted faces, from F before the
// update; a cell still out of bounds is listed for the next round (not in
// the last round, which clips every cell)
__global__ void k_reupdate(DevMesh M, DevState S, double* acc, int64_t risk_cap, bool last) {
  double eb = 0.0, clip = 0.0;
  unsigned long long nclip = 0;
  const int64_t n = min((int64_t)S.cnt[kNRepCells], 2 * S.rep_cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    bool risky = false;
    int64_t c = 0;
    double fn = 0.0, V = 1.0;
    if (i < n) {
      c = S.repc[i];
      const int64_t q0 = M.cf_ptr[c], q1 = M.cf_ptr[c + 1];
      V = M.cvol[c];
      int ni = 0;
      fn = cell_fnext(M, S.tf, S.srate, cell_gdt(M, S.gp, q0, q1), S.VF, S.fexact, q0, q1,
                      S.Fprev[c], V, &ni);
      risky = !last && at_risk(fn, ni);
    }
    const bool listed = warp_append_cap(risky, (int32_t)c, S.risk, S.cnt + kNRisk, risk_cap);
    if (i < n) {
      if (listed) {
        S.F[c] = fn;
      } else {
        eb = fmax(eb, fmax(-V * fn, V * (fn - 1.0)));
        const double fc = fmax(fmin(fn, 1.0), 0.0);
        clip += V * (fn - fc);
        nclip += fc != fn;
        S.F[c] = fc;
      }
    }
  }
  const double s1 = block_sum(clip);
  if (threadIdx.x == 0) acc[kAccClip * kAccSlots + blockIdx.x] += s1;
  for (int o = 16; o > 0; o >>= 1) nclip += __shfl_xor_sync(GVOF_FULL, nclip, o);
  if ((threadIdx.x & 31) == 0 && nclip) atomicAdd(S.cnt + kNClipped, nclip);
  block_ebound(eb, S.red, true);
}

// end of the repair: clip any listed cell still outside [0, 1] (a cell whose
// repair faces did not fit the list), each once, and sum the boundary
// outflow with the final face volumes
__global__ void k_repair_finish(DevMesh M, DevState S, const int32_t* bfaces, int64_t nbf,
                                double* acc, int64_t risk_cap) {
  const int32_t mark = (int32_t)S.cnt[kEpoch] * 16 + 15;
  double eb = 0.0, clip = 0.0, bnd = 0.0;
  unsigned long long nclip = 0;
  const int64_t n = min((int64_t)S.cnt[kNRisk], risk_cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = S.risk[i];
    const double f = S.F[c];
    if (!(f < 0.0 || f > 1.0) || !claim(S.stamp_r, c, mark)) continue;
    const double V = M.cvol[c];
    eb = fmax(eb, fmax(-V * f, V * (f - 1.0)));
    const double fc = fmax(fmin(f, 1.0), 0.0);
    clip += V * (f - fc);
    ++nclip;
    S.F[c] = fc;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbf; i += stride) {
    const int f = bfaces[i];
    const int8_t t = S.tf[f];
    if (t == -1) continue;
    const double vd = S.srate[f] * grid_gdt(M, S.gp, f);
    bnd += face_vf(t, vd, S.VF, f);
  }
  const double s1 = block_sum(clip);
  if (threadIdx.x == 0) acc[kAccClip * kAccSlots + blockIdx.x] += s1;
  const double s2 = block_sum(bnd);
  if (threadIdx.x == 0) acc[kAccBoundary * kAccSlots + blockIdx.x] += s2;
  for (int o = 16; o > 0; o >>= 1) nclip += __shfl_xor_sync(GVOF_FULL, nclip, o);
  if ((threadIdx.x & 31) == 0 && nclip) atomicAdd(S.cnt + kNClipped, nclip);
  block_ebound(eb, S.red, true);
}

// sum of V F in a fixed order: per-block partials then one block
__global__ void k_volume_partial(DevMesh M, const double* F, double* red) {
  double acc = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < M.nc;
       c += (int64_t)gridDim.x * blockDim.x)
    acc += M.cvol[c] * F[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(GVOF_FULL, acc, o);
  __shared__ double s[32];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) s[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s[i];
    red[blockIdx.x] = t;
  }
}

__global__ void k_volume_final(double* red, int nblocks, int neb, const double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nblocks; ++i) t += red[i];
  double eb = 0.0;
  for (int i = 0; i < neb; ++i) eb = fmax(eb, red[kRedSlots / 2 + i]);
  red[kRedSlots - 2] = t;
  red[kRedSlots - 1] = eb;
  for (int a = 0; a < kNAcc; ++a) {
    double s = 0.0;
    for (int i = 0; i < kAccSlots; ++i) s += acc[a * kAccSlots + i];
    red[kRedSlots - 5 + a] = s;
  }
}

constexpr int kUpdBlocks = kSMs * 4;  // fixed, <= kRedSlots/2 - 2

}  // namespace

cudaError_t launch_cell_tags(const vof_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->cnt + kNIcells, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const double eps = c->opt.eps, ome = 1.0 - c->opt.eps;
  long long eb, ob;
  std::memcpy(&eb, &eps, sizeof eb);
  std::memcpy(&ob, &ome, sizeof ob);
  k_cell_tags<<<grid_for(c->nc, 256), 256, 0, s>>>(c->nc, eb, ob, c->F, c->cvol, c->tc, c->icells,
                                                   c->cnt, c->acc + kAccCutoff * kAccSlots,
                                                   c->bcells);
  return cudaGetLastError();
}

cudaError_t launch_node_tags(const vof_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->cnt + kNBandNodes, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_band_nodes<<<kSMs * 4, 256, 0, s>>>(mesh_view(c), c->bcells, c->cnt, c->stamp_v, c->bnodes);
  if (c->opt.precision == VOF_PREC_MIXED)
    k_node_tags<float><<<grid_for(c->nv, 256), 256, 0, s>>>(mesh_view(c), c->F, c->opt.eps, c->tv,
                                                            c->cnt, c->bnodes);
  else
    k_node_tags<double><<<grid_for(c->nv, 256), 256, 0, s>>>(mesh_view(c), c->F, c->opt.eps, c->tv,
                                                             c->cnt, c->bnodes);
  k_band_end<<<1, 32, 0, s>>>(c->cnt);
  return cudaGetLastError();
}

cudaError_t launch_face_sweep(const vof_ctx* c, cudaStream_t s) {
  // counters of this advect: active faces, truncations, overflow, fallbacks
  static_assert(kNAfaces + 1 == kNTrunc && kNTrunc + 3 == kNEdgeOn, "counter layout");
  cudaError_t e = cudaMemsetAsync(c->cnt + kNAfaces, 0, 5 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  // clip, escape and repair counters of this advect
  static_assert(kNClipped + 8 == kNCnt, "counter layout");
  e = cudaMemsetAsync(c->cnt + kNClipped, 0, 8 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_band_begin<<<1, 32, 0, s>>>(c->cnt);
  k_face_sweep<<<grid_for(c->nf, 256), 256, 0, s>>>(mesh_view(c), c->tv, c->tf, c->afaces, c->cnt,
                                                    c->vf_ptr, c->vf, c->bnodes, c->stamp_f);
  return cudaGetLastError();
}
cudaError_t launch_set_fraction(const vof_ctx* c, const double* Fin, cudaStream_t s) {
  k_set_fraction<<<kSMs * 8, 256, 0, s>>>(c->nc, Fin, c->F, c->stamp_c, c->cnt);
  return cudaGetLastError();
}
cudaError_t launch_face_flux_export(const vof_ctx* c, cudaStream_t s) {
  k_face_flux_export<<<grid_for(c->nf, 256), 256, 0, s>>>(mesh_view(c), c->tf, c->srate, c->gp_d,
                                                          c->Vd, c->VF);
  return cudaGetLastError();
}

cudaError_t launch_update(const vof_ctx* c, cudaStream_t s) {
  k_band_cells<<<kUpdBlocks, 256, 0, s>>>(mesh_view(c), c->afaces, c->icells, c->cnt, c->stamp_c,
                                          c->bcells);
  k_update<<<kUpdBlocks, 256, 0, s>>>(mesh_view(c), state_view(c), c->bfaces, c->nbf, c->acc,
                                      c->bcells, c->nc, c->opt.precision == VOF_PREC_MIXED);
  return cudaGetLastError();
}

int repair_launch_count() { return 5 * kRepairRounds + 1; }

cudaError_t launch_repair(const vof_ctx* c, cudaStream_t s) {
  const DevMesh m = mesh_view(c);
  const DevState st = state_view(c);
  for (int r = 1; r <= kRepairRounds; ++r) {
    k_repair_begin<<<1, 32, 0, s>>>(c->cnt, c->nc, c->rep_cap);
    k_risk_cells<<<kSMs * 2, 256, 0, s>>>(m, st, c->stamp_f, c->Eexc, c->Sroom, r);
    k_adjust_faces<<<kSMs * 2, 256, 0, s>>>(m, st, c->Eexc, c->Sroom, r);
    k_repair_cells<<<kSMs * 2, 256, 0, s>>>(m, st, r);
    k_reupdate<<<kUpdBlocks, 256, 0, s>>>(m, st, c->acc, c->nc, r == kRepairRounds);
  }
  k_repair_finish<<<kUpdBlocks, 256, 0, s>>>(m, st, c->bfaces, c->nbf, c->acc, c->nc);
  return cudaGetLastError();
}

cudaError_t launch_volume_sum(const vof_ctx* c, cudaStream_t s) {
  k_volume_partial<<<kUpdBlocks, 256, 0, s>>>(mesh_view(c), c->F, c->red);
  k_volume_final<<<1, 32, 0, s>>>(c->red, kUpdBlocks, kUpdBlocks, c->acc);
  return cudaGetLastError();
}

}  // namespace gvof

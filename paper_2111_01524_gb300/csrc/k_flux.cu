// Face fluxes of the active faces (Sec. 2.2): FMFPA (Sec. 2.2.2), EMFPA
// (Sec. 2.2.1) or NMFPA (Sec. 2.2.3) flux polyhedron of each tag-0 face,
// truncated by the half-spaces of every
// overlapped candidate cell and, for interfacial cells, by its PLIC
// half-space (Sec. 2.2); the truncated volume is a divergence-theorem sum
// over the faces of the clipped polyhedron. One warp per active face.
//
// GPU design of the truncation. The flux polyhedron may be non-convex with
// self-intersecting faces, so it is clipped as a closed oriented surface
// (face loops over a shared vertex table), never decomposed:
//  - every vertex is classified once per plane (inside: a.x + b >= 0), so
//    the two faces sharing an edge always agree on where it is cut;
//  - each face loop is clipped by one lane (Sutherland-Hodgman); the new
//    vertex of a cut edge is created by the face that leaves the half-space
//    along it and looked up by the face that enters along it (key: inside
//    vertex, outside vertex), so it exists once;
//  - the cap is closed topologically: in each face the clipped loop runs
//    exit -> entry along the plane, and the reversed pairs link the new
//    vertices into one or more cap loops. Any pairing of exits and entries
//    along a face is valid for the divergence sum (winding-number
//    semantics), so non-convex and self-intersecting faces need no sorting.
// Shared memory per warp holds the vertex table, two face-loop buffers
// (ping-pong, stored slot-major so that the lanes of a warp read
// consecutive bytes), and the base polyhedron restored per candidate cell.
// Candidate cells are streamed 32 at a time and filtered by tag and by an
// exact bounding-box test in the face-local frame.
// FP64 path: G = double. Mixed path: G = float in face-local coordinates
// scaled by 1/sqrt(A_face), with absolute positions held as (hi, lo) float
// pairs, so no FP64 instruction is executed per truncation.
#include "vof_common.cuh"

namespace gvof {
namespace {

#ifndef GVOF_FLUX_MINB
#define GVOF_FLUX_MINB 8
#endif
// call structure of the flux kernel (inlining trades instruction-cache
// footprint against call overhead and the registers a call saves to local
// memory); chosen by measurement on the 256^3 deformation, mixed: inlining
// the plane truncation, the per-cell truncation, the clip and the streaming
// cut and the per-face routines while the FP64 volume sum, the compaction
// and the non-convex cells stay real calls was fastest (the clip and cut as
// calls: +15%; the per-cell truncation too: +22%; the plane truncation too:
// +48%; a register cap of 72 or 85 instead of 64: +7% and +21%)
#ifndef GVOF_OUTLINE_PLANES
#define GVOF_INLINE_PLANES
#endif
#ifndef GVOF_OUTLINE_OUTER
#define GVOF_INLINE_OUTER
#endif
#ifndef GVOF_OUTLINE_CELL
#define GVOF_INLINE_CELL
#endif
#ifndef GVOF_OUTLINE_CLIP
#define GVOF_INLINE_CLIP
#endif
#ifdef GVOF_INLINE_PLANES
#define GVOF_PLANES_ATTR __forceinline__
#else
#define GVOF_PLANES_ATTR __noinline__
#endif
#ifdef GVOF_INLINE_OUTER
#define GVOF_OUTER_ATTR __forceinline__
#else
#define GVOF_OUTER_ATTR __noinline__
#endif
#ifdef GVOF_INLINE_CLIP
#define GVOF_CLIP_ATTR __forceinline__
#else
#define GVOF_CLIP_ATTR __noinline__
#endif
#ifdef GVOF_INLINE_CELL
#define GVOF_CELL_ATTR __forceinline__
#else
#define GVOF_CELL_ATTR __noinline__
#endif

constexpr int kWarps = 4;
constexpr int MAXI = kMaxFaceVerts;   // face vertices
// base polyhedron vertices: 2I+1 (FMFPA, I <= 8) or 3I+1 (EMFPA, I <= 6)
constexpr int NB = VOF_MAX_POLY_VERTS;
constexpr int NR = 32;                // new vertices per clip

// A flux polyhedron is worked on by a group of GW lanes: a whole warp (GW =
// 32), or half of one (GW = 16: two faces per warp, for polyhedra of at
// most 16 base vertices and face loops against convex cells of at most 16
// faces, which is every hex and tetrahedral grid). Capacities per group:
// vertex table, face loops (one lane each), loop length.
template <typename G, int GW = 32>
struct __align__(16) Poly {
  static constexpr int NV = GW == 32 ? 80 : 64;
  static constexpr int NF = GW;
  static constexpr int LM = GW == 32 ? 32 : 24;
  G vx[NV], vy[NV], vz[NV];
  G phi[NV];
  G bx[NB], by[NB], bz[NB];  // base polyhedron
  uint8_t fv[2][LM][NF];     // loop slot k of face f at fv[buf][k][f]
  uint8_t flen[2][NF];
  uint8_t ra[NR], rb[NR];    // cut-edge records: inside vertex, outside vertex
  int8_t capnext[NR];
  int8_t rnext[NR];          // next record of the same inside vertex
  int rfirst[NV];            // first record of each inside vertex (-1: none)
  uint8_t newid[NV];
  G pl[NF + 1][4];           // half-spaces of the current candidate cell; [NF]: PLIC
  int32_t cand[sizeof(G) == 4 ? 128 : 1];  // candidate cells met by the box of P (FP32)
};

// warp primitives over the lane group of the calling thread (the group's
// lanes are consecutive and aligned: threadIdx.x & 16 is the first lane of
// a half warp); ballots are returned in the group's own lane numbering
template <int GW>
__device__ __forceinline__ unsigned gmask() {
  return GW == 32 ? GVOF_FULL : (0xffffu << (threadIdx.x & 16));
}
template <int GW>
__device__ __forceinline__ unsigned gballot(bool p) {
  if constexpr (GW == 32) return __ballot_sync(GVOF_FULL, p);
  else return (__ballot_sync(gmask<GW>(), p) >> (threadIdx.x & 16)) & 0xffffu;
}
template <int GW>
__device__ __forceinline__ bool gany(bool p) { return __any_sync(gmask<GW>(), p); }
template <int GW, typename T>
__device__ __forceinline__ T gshfl(T v, int src) { return __shfl_sync(gmask<GW>(), v, src, GW); }
template <int GW, typename T>
__device__ __forceinline__ T gshfl_up(T v, int d) { return __shfl_up_sync(gmask<GW>(), v, d, GW); }
// sum over the group's lanes: a butterfly from GW/2 down; lanes that hold
// 0 leave the others' partial sums exact, so a whole warp whose upper half
// holds 0 sums as a half warp does, bit for bit
template <int GW, typename T>
__device__ __forceinline__ T gsum(T v) {
  for (int o = GW / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask<GW>(), v, o);
  return v;
}
template <int GW>
__device__ __forceinline__ void gsync() { __syncwarp(gmask<GW>()); }
template <typename G>
__host__ __device__ constexpr int cand_cap() { return sizeof(G) == 4 ? 128 : 0; }

__device__ __forceinline__ double absval(double a) { return a; }
__device__ __forceinline__ float absval(float2 a) { return a.x + a.y; }
__device__ __forceinline__ double absd(double a) { return a; }
__device__ __forceinline__ double absd(float2 a) { return (double)a.x + (double)a.y; }

struct PolyState {
  int nv, nf, cur;
};

// vertices of the base polyhedron of a face of I nodes
template <int KIND>
__device__ __forceinline__ int base_verts(int I) {
  return KIND == VOF_FLUX_EMFPA ? 3 * I + 1 : KIND == VOF_FLUX_NMFPA ? 2 * I : 2 * I + 1;
}

// restore the base polyhedron from P.b*.
// FMFPA (Sec. 2.2.2): x_0..x_{I-1}, back-traced I..2I-1, apex 2I; faces: the
// cell face, I side quads, I bottom triangles. A side quad whose
// back-traced vertices do not both lie on its side plane (streak-line
// fallback) is not planar; it is split into the triangles (x_{i+1}, x_i,
// x_{I+i}) and (x_{i+1}, x_{I+i}, x_{I+i+1}), bit i of split.
// EMFPA (Sec. 2.2.1): the same first 2I vertices, side-face centres
// 2I..3I-1, apex 3I; faces: the cell face, four triangles per side quad
// (x_{i+1}, x_i, x_{I+i}, x_{I+i+1}) joining its edges to its centre, I
// bottom triangles.
// NMFPA (Sec. 2.2.3): the first 2I vertices only; faces: the cell face, I
// planar side quads, the back-traced face (reversed: its normal is -n).
template <typename G, int KIND, int GW>
__device__ void restore_base(Poly<G, GW>& P, PolyState& st, int I, unsigned split, int lane) {
  if constexpr (KIND == VOF_FLUX_NMFPA) {
    const int nvb = 2 * I;
    if (lane < nvb) { P.vx[lane] = P.bx[lane]; P.vy[lane] = P.by[lane]; P.vz[lane] = P.bz[lane]; }
    if (lane == 0) {
      for (int i = 0; i < I; ++i) P.fv[0][i][0] = (uint8_t)i;
      P.flen[0][0] = (uint8_t)I;
    } else if (lane <= I) {
      const int i = lane - 1, ip = (i + 1 == I) ? 0 : i + 1;
      P.fv[0][0][lane] = (uint8_t)ip;
      P.fv[0][1][lane] = (uint8_t)i;
      P.fv[0][2][lane] = (uint8_t)(I + i);
      P.fv[0][3][lane] = (uint8_t)(I + ip);
      P.flen[0][lane] = 4;
    } else if (lane == I + 1) {
      for (int i = 0; i < I; ++i) P.fv[0][i][lane] = (uint8_t)(2 * I - 1 - i);
      P.flen[0][lane] = (uint8_t)I;
    }
    st.nv = nvb;
    st.nf = I + 2;
    st.cur = 0;
    gsync<GW>();
    return;
  } else if constexpr (KIND == VOF_FLUX_EMFPA) {
    const int nvb = 3 * I + 1, nfb = 5 * I + 1;
    if (lane < nvb) { P.vx[lane] = P.bx[lane]; P.vy[lane] = P.by[lane]; P.vz[lane] = P.bz[lane]; }
    if (lane == 0) {
      for (int i = 0; i < I; ++i) P.fv[0][i][0] = (uint8_t)i;
      P.flen[0][0] = (uint8_t)I;
    } else if (lane <= 4 * I) {
      const int t = lane - 1, i = t >> 2, e = t & 3, ip = (i + 1 == I) ? 0 : i + 1;
      // edge e of the side quad (ip, i, I+i, I+ip), then its centre
      const int a = e == 0 ? ip : e == 1 ? i : e == 2 ? I + i : I + ip;
      const int b = e == 0 ? i : e == 1 ? I + i : e == 2 ? I + ip : ip;
      P.fv[0][0][lane] = (uint8_t)a;
      P.fv[0][1][lane] = (uint8_t)b;
      P.fv[0][2][lane] = (uint8_t)(2 * I + i);
      P.flen[0][lane] = 3;
    } else if (lane < nfb) {
      const int i = lane - 1 - 4 * I, ip = (i + 1 == I) ? 0 : i + 1;
      P.fv[0][0][lane] = (uint8_t)(I + ip);
      P.fv[0][1][lane] = (uint8_t)(I + i);
      P.fv[0][2][lane] = (uint8_t)(3 * I);
      P.flen[0][lane] = 3;
    }
    st.nv = nvb;
    st.nf = nfb;
    st.cur = 0;
    gsync<GW>();
    return;
  } else {
  const int nvb = 2 * I + 1;
  const int nsplit = __popc(split);
  if (lane < nvb) {
    P.vx[lane] = P.bx[lane]; P.vy[lane] = P.by[lane]; P.vz[lane] = P.bz[lane];
    if (lane == 0) {
      for (int i = 0; i < I; ++i) P.fv[0][i][0] = (uint8_t)i;
      P.flen[0][0] = (uint8_t)I;
    } else if (lane <= I) {
      const int i = lane - 1, ip = (i + 1 == I) ? 0 : i + 1;
      const int slot = 1 + i + __popc(split & ((1u << i) - 1u));
      if ((split >> i) & 1u) {
        P.fv[0][0][slot] = (uint8_t)ip;
        P.fv[0][1][slot] = (uint8_t)i;
        P.fv[0][2][slot] = (uint8_t)(I + i);
        P.flen[0][slot] = 3;
        P.fv[0][0][slot + 1] = (uint8_t)ip;
        P.fv[0][1][slot + 1] = (uint8_t)(I + i);
        P.fv[0][2][slot + 1] = (uint8_t)(I + ip);
        P.flen[0][slot + 1] = 3;
      } else {
        P.fv[0][0][slot] = (uint8_t)ip;
        P.fv[0][1][slot] = (uint8_t)i;
        P.fv[0][2][slot] = (uint8_t)(I + i);
        P.fv[0][3][slot] = (uint8_t)(I + ip);
        P.flen[0][slot] = 4;
      }
    } else {
      const int i = lane - 1 - I, ip = (i + 1 == I) ? 0 : i + 1;
      const int slot = lane + nsplit;
      P.fv[0][0][slot] = (uint8_t)(I + ip);
      P.fv[0][1][slot] = (uint8_t)(I + i);
      P.fv[0][2][slot] = (uint8_t)(2 * I);
      P.flen[0][slot] = 3;
    }
  }
  st.nv = nvb;
  st.nf = nvb + nsplit;
  st.cur = 0;
  gsync<GW>();
  }
}

// drop unreferenced vertices and renumber (keeps room for a clip)
template <typename G, int GW>
__device__ __noinline__ void compact(Poly<G, GW>& P, PolyState& st, int lane) {
  constexpr int NV = Poly<G, GW>::NV;
  constexpr int VPL = (NV + GW - 1) / GW;  // vertex slots per lane
  for (int v = lane; v < NV; v += GW) P.newid[v] = 0;
  gsync<GW>();
  if (lane < st.nf) {
    const int L = P.flen[st.cur][lane];
    for (int k = 0; k < L; ++k) P.newid[P.fv[st.cur][k][lane]] = 1;
  }
  gsync<GW>();
  int m[VPL], s = 0;
  for (int r = 0; r < VPL; ++r) {
    const int v = lane * VPL + r;
    m[r] = (v < st.nv) ? P.newid[v] : 0;
    s += m[r];
  }
  int incl = s;
  for (int d = 1; d < GW; d <<= 1) {
    const int t = gshfl_up<GW>(incl, d);
    if (lane >= d) incl += t;
  }
  const int total = gshfl<GW>(incl, GW - 1);
  int base = incl - s;
  G x[VPL], y[VPL], z[VPL];
  for (int r = 0; r < VPL; ++r) {
    const int v = lane * VPL + r;
    if (v < st.nv && m[r]) { x[r] = P.vx[v]; y[r] = P.vy[v]; z[r] = P.vz[v]; }
  }
  gsync<GW>();
  for (int r = 0; r < VPL; ++r) {
    const int v = lane * VPL + r;
    if (v < st.nv && m[r]) {
      P.vx[base] = x[r]; P.vy[base] = y[r]; P.vz[base] = z[r];
      P.newid[v] = (uint8_t)base;
      ++base;
    }
  }
  gsync<GW>();
  if (lane < st.nf) {
    const int L = P.flen[st.cur][lane];
    for (int k = 0; k < L; ++k) P.fv[st.cur][k][lane] = P.newid[P.fv[st.cur][k][lane]];
  }
  st.nv = total;
  gsync<GW>();
}

// clip the closed surface by the half-space a.x + b >= 0.
// returns 0: unchanged, 1: clipped, 2: empty. err bit0: capacity overflow
// or inconsistent topology (the face's V_F is then unreliable and counted).
template <typename G, int GW>
__device__ GVOF_CLIP_ATTR int clip(Poly<G, GW>& P, PolyState& st, G a0, G a1, G a2, G b, int lane,
                                 unsigned& err) {
  constexpr int NV = Poly<G, GW>::NV, NF = Poly<G, GW>::NF, LM = Poly<G, GW>::LM;
  if (st.nv > NV - NR) compact(P, st, lane);
  bool vout = false;
  for (int v = lane; v < st.nv; v += GW) {
    const G ph = a0 * P.vx[v] + a1 * P.vy[v] + a2 * P.vz[v] + b;
    P.phi[v] = ph;
    P.rfirst[v] = -1;
    vout |= !(ph >= G(0));
  }
  if (!gany<GW>(vout)) return 0;  // no vertex outside: unchanged
  gsync<GW>();
  const int cur = st.cur, nf = st.nf, nv = st.nv;
  const int fl = lane < NF ? lane : 0;
  bool has_in = false, has_out = false;
  int nexit = 0, L = 0;
  unsigned inmask = 0u;  // bit k: loop vertex k inside
  if (lane < nf) {
    L = P.flen[cur][lane];
    for (int k = 0; k < L; ++k)
      if (P.phi[P.fv[cur][k][fl]] >= G(0)) inmask |= 1u << k;
    const unsigned full = (L == 32) ? 0xffffffffu : ((1u << L) - 1u);
    has_in = inmask != 0u;
    has_out = inmask != full;
    // exit edges k -> k+1: k inside, k+1 outside
    const unsigned nxt_in = ((inmask >> 1) | (inmask << (L - 1))) & full;
    nexit = __popc(inmask & ~nxt_in);
  }
  const unsigned bin = gballot<GW>(has_in);
  const unsigned bout = gballot<GW>(has_out);
  if (bout == 0) return 0;
  if (bin == 0) { st.nf = 0; return 2; }
  int incl = nexit;
  for (int d = 1; d < GW; d <<= 1) {
    const int t = gshfl_up<GW>(incl, d);
    if (lane >= d) incl += t;
  }
  const int total = gshfl<GW>(incl, GW - 1);
  const int off = incl - nexit;
  if (total > NR || nv + total > NV) { err |= 1u; st.nf = 0; return 2; }
  // new vertices on the cut edges, created by the face leaving the half-space
  if (lane < nf && nexit) {
    int r = off;
    for (int k = 0; k < L; ++k) {
      const int k1 = (k + 1 == L) ? 0 : k + 1;
      if (((inmask >> k) & 1u) && !((inmask >> k1) & 1u)) {
        const int va = P.fv[cur][k][fl], vb = P.fv[cur][k1][fl];
        const G pa = P.phi[va], pb = P.phi[vb];
        const G t = pa / (pa - pb);
        const int id = nv + r;
        P.vx[id] = P.vx[va] + t * (P.vx[vb] - P.vx[va]);
        P.vy[id] = P.vy[va] + t * (P.vy[vb] - P.vy[va]);
        P.vz[id] = P.vz[va] + t * (P.vz[vb] - P.vz[va]);
        P.ra[r] = (uint8_t)va;
        P.rb[r] = (uint8_t)vb;
        P.capnext[r] = -1;
        P.rnext[r] = (int8_t)atomicExch(&P.rfirst[va], r);  // chain by inside vertex
        ++r;
      }
    }
  }
  gsync<GW>();
  const int nxt = cur ^ 1;
  const int slot = __popc(bin & ((1u << lane) - 1u));
  bool bad = false;
  if (lane < nf && has_in) {
    const int k0 = __ffs(inmask) - 1;
    int n = 0, pend = -1;
    for (int s = 0; s < L; ++s) {
      int k = k0 + s;
      if (k >= L) k -= L;
      const int k1 = (k + 1 == L) ? 0 : k + 1;
      const int va = P.fv[cur][k][fl];
      const bool ia = (inmask >> k) & 1u, ib = (inmask >> k1) & 1u;
      if (ia) {
        if (n < LM) P.fv[nxt][n][slot] = (uint8_t)va;
        ++n;
      }
      if (ia != ib) {
        const int vb = P.fv[cur][k1][fl];
        // record of the cut edge (inside vertex, outside vertex)
        const int vin = ia ? va : vb, vout2 = ia ? vb : va;
        int r = P.rfirst[vin];
        while (r >= 0 && P.rb[r] != vout2) r = P.rnext[r];
        if (r < 0 || (!ia && pend < 0)) { bad = true; break; }
        if (n < LM) P.fv[nxt][n][slot] = (uint8_t)(nv + r);
        ++n;
        if (ia) pend = r;
        else P.capnext[r] = (int8_t)pend;  // cap edge: entry -> preceding exit
      }
    }
    if (n > LM) bad = true;
    P.flen[nxt][slot] = (uint8_t)(n > LM ? LM : n);
  }
  if (gany<GW>(bad)) { err |= 1u; st.nf = 0; return 2; }
  gsync<GW>();
  // cap loops
  int nfo = __popc(bin);
  if (lane == 0) {
    unsigned vis = 0u;
    for (int r = 0; r < total; ++r) {
      if ((vis >> r) & 1u) continue;
      if (nfo >= NF) { err |= 1u; break; }
      int n = 0, s = r;
      while (s >= 0 && !((vis >> s) & 1u) && n < LM) {
        vis |= 1u << s;
        P.fv[nxt][n++][nfo] = (uint8_t)(nv + s);
        s = P.capnext[s];
      }
      if (s != r) err |= 1u;  // open chain: inconsistent topology
      if (n >= 3) { P.flen[nxt][nfo] = (uint8_t)n; ++nfo; }
    }
  }
  nfo = gshfl<GW>(nfo, 0);
  st.nv = nv + total;
  st.nf = nfo;
  st.cur = nxt;
  gsync<GW>();
  return 1;
}

// signed volume of the surface: each lane fans one face loop
template <typename G, int GW>
__device__ __noinline__ G volume(const Poly<G, GW>& P, const PolyState& st, int lane) {
  G acc = G(0);
  if (st.nf > 0) {
    const int o = P.fv[st.cur][0][0];
    const G ox = P.vx[o], oy = P.vy[o], oz = P.vz[o];
    if (lane < st.nf) {
      const int L = P.flen[st.cur][lane];
      const int i0 = P.fv[st.cur][0][lane], i1 = P.fv[st.cur][1][lane];
      const G x0 = P.vx[i0] - ox, y0 = P.vy[i0] - oy, z0 = P.vz[i0] - oz;
      G px = P.vx[i1] - ox, py = P.vy[i1] - oy, pz = P.vz[i1] - oz;
      for (int k = 2; k < L; ++k) {
        const int ik = P.fv[st.cur][k][lane];
        const G qx = P.vx[ik] - ox, qy = P.vy[ik] - oy, qz = P.vz[ik] - oz;
        acc += x0 * (py * qz - pz * qy) + y0 * (pz * qx - px * qz) + z0 * (px * qy - py * qx);
        px = qx; py = qy; pz = qz;
      }
    }
  }
  return gsum<GW>(acc) / G(6);
}

// volume of the part of the surface on the inner side a.x + b >= 0 of a
// plane, without building the cut: each lane clips its face loop on the fly
// (Sutherland-Hodgman) and fans it with the origin ON the plane, so the cap
// the cut would close contributes nothing to the divergence sum
template <typename G, int GW>
__device__ GVOF_CLIP_ATTR G volume_cut(const Poly<G, GW>& P, const PolyState& st, G a0, G a1, G a2, G b,
                                     int lane) {
  // origin: projection onto the plane of a vertex on the inner side, so that
  // the fan terms are of the size of the part that is kept (which may be a
  // thin sliver of the polyhedron) and the FP32 error scales with it
  int myv = -1;
  if (lane < st.nf) {
    const int L = P.flen[st.cur][lane];
    for (int k = 0; k < L; ++k) {
      const int v = P.fv[st.cur][k][lane];
      if (a0 * P.vx[v] + a1 * P.vy[v] + a2 * P.vz[v] + b >= G(0)) { myv = v; break; }
    }
  }
  const unsigned have = gballot<GW>(myv >= 0);
  if (have == 0u) return G(0);  // no vertex on the inner side: nothing is kept
  const int v0 = gshfl<GW>(myv, __ffs(have) - 1);
  G acc = G(0);
  if (lane < st.nf) {
    const G aa = a0 * a0 + a1 * a1 + a2 * a2;
    const G d0 = (a0 * P.vx[v0] + a1 * P.vy[v0] + a2 * P.vz[v0] + b) / aa;
    const G ox = P.vx[v0] - d0 * a0, oy = P.vy[v0] - d0 * a1, oz = P.vz[v0] - d0 * a2;
    const int L = P.flen[st.cur][lane];
    int v = P.fv[st.cur][L - 1][lane];
    G ax = P.vx[v] - ox, ay = P.vy[v] - oy, az = P.vz[v] - oz;
    G pa = a0 * ax + a1 * ay + a2 * az;
    int ne = 0;
    G q0x = 0, q0y = 0, q0z = 0, qpx = 0, qpy = 0, qpz = 0;
    for (int k = 0; k < L; ++k) {
      v = P.fv[st.cur][k][lane];
      const G bx = P.vx[v] - ox, by = P.vy[v] - oy, bz = P.vz[v] - oz;
      const G pb = a0 * bx + a1 * by + a2 * bz;
      const bool ia = pa >= G(0), ib = pb >= G(0);
      for (int e = 0; e < 2; ++e) {
        G px, py, pz;
        if (e == 0) {
          if (ia == ib) continue;
          // interpolate from the inside end, as the face on the other side of
          // this edge does, so both compute the same point bit for bit
          if (ia) {
            const G t = pa / (pa - pb);
            px = ax + t * (bx - ax); py = ay + t * (by - ay); pz = az + t * (bz - az);
          } else {
            const G t = pb / (pb - pa);
            px = bx + t * (ax - bx); py = by + t * (ay - by); pz = bz + t * (az - bz);
          }
        } else {
          if (!ib) continue;
          px = bx; py = by; pz = bz;
        }
        if (ne == 0) { q0x = px; q0y = py; q0z = pz; }
        else if (ne >= 2)
          acc += q0x * (qpy * pz - qpz * py) + q0y * (qpz * px - qpx * pz) + q0z * (qpx * py - qpy * px);
        qpx = px; qpy = py; qpz = pz;
        ++ne;
      }
      ax = bx; ay = by; az = bz; pa = pb;
    }
  }
  return gsum<GW>(acc) / G(6);
}

template <typename G>
struct FaceFrame {
  typename Prec<G>::A cx, cy, cz;  // face centroid (absolute)
  G L, sc;                         // sqrt(A), 1/sqrt(A)
  int I;
  G lo[3], hi[3];                  // local bounding box of the polyhedron
  int degenerate, edgeon;
  unsigned split;                  // non-planar FMFPA side quads (bit i: side i)
};

// FMFPA construction (Sec. 2.2.2) by one thread: side plane i contains
// edge i and is parallel to the velocity at the edge centre; back-traced
// vertex i is the projection of the streak-line point x_i - dt u_i (Eq.
// streak-line2) on the line where side planes i-1 and i meet (the
// streak-line point itself where that line or a plane is ill-conditioned,
// sin < 1e-3); the centroid of the back-traced loop moves along the face
// normal by the closed-form amount that makes the signed volume equal V_d.
// Writes the 2I+1 vertices (face-local, scaled by 1/sqrt(A)) to v* and the
// frame to fr. One thread per face, so that a warp builds 32 polyhedra at
// once (the construction has one vertex per lane otherwise, 4 of 32 busy for
// a hex face); the flux kernel, its fallback and the polyhedron export all
// use this same arithmetic.
template <typename G>
__device__ __noinline__ bool fmfpa_scalar(const DevMesh& M, const GeoView<G>& Gv, const GridParam& p, int j,
                             double Vd, G* vx, G* vy, G* vz, FaceFrame<G>& fr) {
  const int64_t fb = M.fptr[j];
  const int I = (int)(M.fptr[j + 1] - fb);
  fr.I = I;
  fr.degenerate = 0;
  fr.edgeon = 0;
  fr.split = 0u;
  if (I > MAXI || I < 3) return false;
  fr.cx = Gv.fcx[j]; fr.cy = Gv.fcy[j]; fr.cz = Gv.fcz[j];
  fr.L = sqrt(Gv.fa[j]);
  fr.sc = G(1) / fr.L;
  const G nx = Gv.fnx[j], ny = Gv.fny[j], nz = Gv.fnz[j];
  const G k = (G)(p.g * p.dt) * fr.sc;
  G lx[MAXI], ly[MAXI], lz[MAXI], ax[MAXI], ay[MAXI], az[MAXI], ux[MAXI], uy[MAXI], uz[MAXI];
  for (int i = 0; i < I; ++i) {
    const int vi = M.fvert[fb + i];
    const typename Prec<G>::A X = Gv.vx[vi], Y = Gv.vy[vi], Z = Gv.vz[vi];
    ax[i] = absval(X); ay[i] = absval(Y); az[i] = absval(Z);
    vel0<G>(p.vel, ax[i], ay[i], az[i], ux[i], uy[i], uz[i]);
    ux[i] *= k; uy[i] *= k; uz[i] *= k;
    lx[i] = rel(X, fr.cx) * fr.sc; ly[i] = rel(Y, fr.cy) * fr.sc; lz[i] = rel(Z, fr.cz) * fr.sc;
  }
  // side plane normal s_i = e_i x u_e,i, with the norms of s, e and u_e
  G sx[MAXI], sy[MAXI], sz[MAXI], ns[MAXI], ne[MAXI], nue[MAXI];
  for (int i = 0; i < I; ++i) {
    const int n = (i + 1 >= I) ? 0 : i + 1;
    G eux, euy, euz;
    vel0<G>(p.vel, G(0.5) * (ax[i] + ax[n]), G(0.5) * (ay[i] + ay[n]), G(0.5) * (az[i] + az[n]), eux,
            euy, euz);
    eux *= k; euy *= k; euz *= k;
    const G ex = lx[n] - lx[i], ey = ly[n] - ly[i], ez = lz[n] - lz[i];
    sx[i] = ey * euz - ez * euy; sy[i] = ez * eux - ex * euz; sz[i] = ex * euy - ey * eux;
    ns[i] = sqrt(sx[i] * sx[i] + sy[i] * sy[i] + sz[i] * sz[i]);
    ne[i] = sqrt(ex * ex + ey * ey + ez * ez);
    nue[i] = sqrt(eux * eux + euy * euy + euz * euz);
  }
  const G tol = (G)1e-3;
  unsigned bad = 0u;
  G bxl[MAXI], byl[MAXI], bzl[MAXI];
  for (int i = 0; i < I; ++i) {
    const int pv = (i == 0) ? I - 1 : i - 1;
    const G dx = sy[pv] * sz[i] - sz[pv] * sy[i], dy = sz[pv] * sx[i] - sx[pv] * sz[i],
            dz = sx[pv] * sy[i] - sy[pv] * sx[i];
    const G dd = dx * dx + dy * dy + dz * dz;
    const bool ok = ns[i] > tol * ne[i] * nue[i] && ns[pv] > tol * ne[pv] * nue[pv] &&
                    sqrt(dd) > tol * ns[pv] * ns[i];
    if (ok) {
      const G kk = (ux[i] * dx + uy[i] * dy + uz[i] * dz) / dd;
      bxl[i] = lx[i] - kk * dx; byl[i] = ly[i] - kk * dy; bzl[i] = lz[i] - kk * dz;
    } else {
      bxl[i] = lx[i] - ux[i]; byl[i] = ly[i] - uy[i]; bzl[i] = lz[i] - uz[i];
      bad |= 1u << i;
    }
  }
  fr.degenerate = __popc(bad);
  // side i joins back-traced vertices i and i+1: planar only if both lie
  // on its side plane
  const unsigned full_mask = (I >= 32) ? 0xffffffffu : ((1u << I) - 1u);
  fr.split = (bad | (((bad >> 1) | (bad << (I - 1))) & full_mask)) & full_mask;
  // centroid of the back-traced loop, its vector area B, and the signed
  // volume with the apex at the centroid (origin = face centroid)
  auto det3 = [](G ax_, G ay_, G az_, G bx_, G by_, G bz_, G cx_, G cy_, G cz_) {
    return ax_ * (by_ * cz_ - bz_ * cy_) + ay_ * (bz_ * cx_ - bx_ * cz_) +
           az_ * (bx_ * cy_ - by_ * cx_);
  };
  const G inv_I = G(1) / (G)I;
  G sxc = 0, syc = 0, szc = 0, Bx = 0, By = 0, Bz = 0;
  for (int i = 0; i < I; ++i) {
    const int n = (i + 1 >= I) ? 0 : i + 1;
    sxc += bxl[i]; syc += byl[i]; szc += bzl[i];
    Bx += G(0.5) * (byl[i] * bzl[n] - bzl[i] * byl[n]);
    By += G(0.5) * (bzl[i] * bxl[n] - bxl[i] * bzl[n]);
    Bz += G(0.5) * (bxl[i] * byl[n] - byl[i] * bxl[n]);
  }
  const G xcx = sxc * inv_I, xcy = syc * inv_I, xcz = szc * inv_I;
  G v6 = G(0);
  for (int i = 0; i < I; ++i) {
    const int n = (i + 1 >= I) ? 0 : i + 1;
    if (i >= 1 && i + 1 < I) v6 += det3(lx[0], ly[0], lz[0], lx[i], ly[i], lz[i], lx[n], ly[n], lz[n]);
    v6 += det3(lx[n], ly[n], lz[n], lx[i], ly[i], lz[i], bxl[i], byl[i], bzl[i]);       // side quad,
    v6 += det3(lx[n], ly[n], lz[n], bxl[i], byl[i], bzl[i], bxl[n], byl[n], bzl[n]);    // fan from x_{i+1}
    v6 += det3(bxl[n], byl[n], bzl[n], bxl[i], byl[i], bzl[i], xcx, xcy, xcz);          // bottom triangle
  }
  const G V0 = v6 / G(6);
  const G Vl = (G)Vd * (fr.sc * fr.sc * fr.sc);
  const G nB = nx * Bx + ny * By + nz * Bz;
  G lam = G(0);
  if (fabs(nB) > G(1e-8)) lam = G(3) * (V0 - Vl) / nB;
  else fr.edgeon = 1;
  for (int i = 0; i < I; ++i) {
    vx[i] = lx[i]; vy[i] = ly[i]; vz[i] = lz[i];
    vx[I + i] = bxl[i]; vy[I + i] = byl[i]; vz[I + i] = bzl[i];
  }
  vx[2 * I] = xcx + lam * nx;
  vy[2 * I] = xcy + lam * ny;
  vz[2 * I] = xcz + lam * nz;
  // local bounding box of the polyhedron
  fr.lo[0] = fr.hi[0] = vx[0]; fr.lo[1] = fr.hi[1] = vy[0]; fr.lo[2] = fr.hi[2] = vz[0];
  for (int v = 1; v <= 2 * I; ++v) {
    fr.lo[0] = min(fr.lo[0], vx[v]); fr.hi[0] = max(fr.hi[0], vx[v]);
    fr.lo[1] = min(fr.lo[1], vy[v]); fr.hi[1] = max(fr.hi[1], vy[v]);
    fr.lo[2] = min(fr.lo[2], vz[v]); fr.hi[2] = max(fr.hi[2], vz[v]);
  }
  return true;
}

// EMFPA construction (Sec. 2.2.1) by one thread: every vertex goes back
// along its own streak line with its own velocity at t^{n+1/2} (Eq.
// streak-line2); side face i (x_i, x_{i+1} and their back-traced points) is
// represented by its vertex-average centre; the centroid of the back-traced
// loop moves along the face normal by the closed-form amount that makes the
// signed volume of the 5I+1 faces equal V_d. Faces sharing an edge compute
// the same four side points from the same two nodes, so their side
// triangles coincide. Vertices: x_0..x_{I-1}, back-traced I..2I-1, side
// centres 2I..3I-1, apex 3I.
template <typename G>
__device__ __noinline__ bool emfpa_scalar(const DevMesh& M, const GeoView<G>& Gv, const GridParam& p, int j,
                                          double Vd, G* vx, G* vy, G* vz, FaceFrame<G>& fr) {
  const int64_t fb = M.fptr[j];
  const int I = (int)(M.fptr[j + 1] - fb);
  fr.I = I;
  fr.degenerate = 0;
  fr.edgeon = 0;
  fr.split = 0u;
  if (I > kMaxEmfpaVerts || I < 3) return false;
  fr.cx = Gv.fcx[j]; fr.cy = Gv.fcy[j]; fr.cz = Gv.fcz[j];
  fr.L = sqrt(Gv.fa[j]);
  fr.sc = G(1) / fr.L;
  const G nx = Gv.fnx[j], ny = Gv.fny[j], nz = Gv.fnz[j];
  const G k = (G)(p.g * p.dt) * fr.sc;
  for (int i = 0; i < I; ++i) {
    const int vi = M.fvert[fb + i];
    const typename Prec<G>::A X = Gv.vx[vi], Y = Gv.vy[vi], Z = Gv.vz[vi];
    G ux, uy, uz;
    vel0<G>(p.vel, absval(X), absval(Y), absval(Z), ux, uy, uz);
    const G lx = rel(X, fr.cx) * fr.sc, ly = rel(Y, fr.cy) * fr.sc, lz = rel(Z, fr.cz) * fr.sc;
    vx[i] = lx; vy[i] = ly; vz[i] = lz;
    vx[I + i] = lx - k * ux; vy[I + i] = ly - k * uy; vz[I + i] = lz - k * uz;
  }
  auto det3 = [](G ax_, G ay_, G az_, G bx_, G by_, G bz_, G cx_, G cy_, G cz_) {
    return ax_ * (by_ * cz_ - bz_ * cy_) + ay_ * (bz_ * cx_ - bx_ * cz_) +
           az_ * (bx_ * cy_ - by_ * cx_);
  };
  const G inv_I = G(1) / (G)I;
  G sxc = 0, syc = 0, szc = 0, Bx = 0, By = 0, Bz = 0;
  for (int i = 0; i < I; ++i) {
    const int n = (i + 1 >= I) ? 0 : i + 1;
    // centre of side face i
    vx[2 * I + i] = G(0.25) * (vx[i] + vx[n] + vx[I + i] + vx[I + n]);
    vy[2 * I + i] = G(0.25) * (vy[i] + vy[n] + vy[I + i] + vy[I + n]);
    vz[2 * I + i] = G(0.25) * (vz[i] + vz[n] + vz[I + i] + vz[I + n]);
    const G bx = vx[I + i], by = vy[I + i], bz = vz[I + i], bxn = vx[I + n], byn = vy[I + n], bzn = vz[I + n];
    sxc += bx; syc += by; szc += bz;
    Bx += G(0.5) * (by * bzn - bz * byn);
    By += G(0.5) * (bz * bxn - bx * bzn);
    Bz += G(0.5) * (bx * byn - by * bxn);
  }
  const G xcx = sxc * inv_I, xcy = syc * inv_I, xcz = szc * inv_I;
  // signed volume with the apex at the centroid (origin = face centroid)
  G v6 = G(0);
  for (int i = 0; i < I; ++i) {
    const int n = (i + 1 >= I) ? 0 : i + 1;
    const G lx = vx[i], ly = vy[i], lz = vz[i], lxn = vx[n], lyn = vy[n], lzn = vz[n];
    const G bx = vx[I + i], by = vy[I + i], bz = vz[I + i], bxn = vx[I + n], byn = vy[I + n], bzn = vz[I + n];
    const G sx = vx[2 * I + i], sy = vy[2 * I + i], sz = vz[2 * I + i];
    if (i >= 1 && i + 1 < I) v6 += det3(vx[0], vy[0], vz[0], lx, ly, lz, lxn, lyn, lzn);
    v6 += det3(lxn, lyn, lzn, lx, ly, lz, sx, sy, sz);  // side triangles
    v6 += det3(lx, ly, lz, bx, by, bz, sx, sy, sz);
    v6 += det3(bx, by, bz, bxn, byn, bzn, sx, sy, sz);
    v6 += det3(bxn, byn, bzn, lxn, lyn, lzn, sx, sy, sz);
    v6 += det3(bxn, byn, bzn, bx, by, bz, xcx, xcy, xcz);  // bottom triangle
  }
  const G V0 = v6 / G(6);
  const G Vl = (G)Vd * (fr.sc * fr.sc * fr.sc);
  const G nB = nx * Bx + ny * By + nz * Bz;
  G lam = G(0);
  if (fabs(nB) > G(1e-8)) lam = G(3) * (V0 - Vl) / nB;
  else fr.edgeon = 1;
  vx[3 * I] = xcx + lam * nx;
  vy[3 * I] = xcy + lam * ny;
  vz[3 * I] = xcz + lam * nz;
  fr.lo[0] = fr.hi[0] = vx[0]; fr.lo[1] = fr.hi[1] = vy[0]; fr.lo[2] = fr.hi[2] = vz[0];
  for (int v = 1; v <= 3 * I; ++v) {
    fr.lo[0] = min(fr.lo[0], vx[v]); fr.hi[0] = max(fr.hi[0], vx[v]);
    fr.lo[1] = min(fr.lo[1], vy[v]); fr.hi[1] = max(fr.hi[1], vy[v]);
    fr.lo[2] = min(fr.lo[2], vz[v]); fr.hi[2] = max(fr.hi[2], vz[v]);
  }
  return true;
}

// NMFPA construction (Sec. 2.2.3) by one thread: every vertex moves back by
// dt times the velocity at the face centre at t^{n+1/2}, so the polyhedron
// is the prism between the face and its translate, of volume V_d by itself
template <typename G>
__device__ __noinline__ bool nmfpa_scalar(const DevMesh& M, const GeoView<G>& Gv, const GridParam& p, int j,
                                          G* vx, G* vy, G* vz, FaceFrame<G>& fr) {
  const int64_t fb = M.fptr[j];
  const int I = (int)(M.fptr[j + 1] - fb);
  fr.I = I;
  fr.degenerate = 0;
  fr.edgeon = 0;
  fr.split = 0u;
  if (I > MAXI || I < 3) return false;
  fr.cx = Gv.fcx[j]; fr.cy = Gv.fcy[j]; fr.cz = Gv.fcz[j];
  fr.L = sqrt(Gv.fa[j]);
  fr.sc = G(1) / fr.L;
  G ux, uy, uz;
  vel0<G>(p.vel, absval(fr.cx), absval(fr.cy), absval(fr.cz), ux, uy, uz);
  const G k = (G)(p.g * p.dt) * fr.sc;
  for (int i = 0; i < I; ++i) {
    const int vi = M.fvert[fb + i];
    const G lx = rel(Gv.vx[vi], fr.cx) * fr.sc, ly = rel(Gv.vy[vi], fr.cy) * fr.sc,
            lz = rel(Gv.vz[vi], fr.cz) * fr.sc;
    vx[i] = lx; vy[i] = ly; vz[i] = lz;
    vx[I + i] = lx - k * ux; vy[I + i] = ly - k * uy; vz[I + i] = lz - k * uz;
  }
  fr.lo[0] = fr.hi[0] = vx[0]; fr.lo[1] = fr.hi[1] = vy[0]; fr.lo[2] = fr.hi[2] = vz[0];
  for (int v = 1; v < 2 * I; ++v) {
    fr.lo[0] = min(fr.lo[0], vx[v]); fr.hi[0] = max(fr.hi[0], vx[v]);
    fr.lo[1] = min(fr.lo[1], vy[v]); fr.hi[1] = max(fr.hi[1], vy[v]);
    fr.lo[2] = min(fr.lo[2], vz[v]); fr.hi[2] = max(fr.hi[2], vz[v]);
  }
  return true;
}

// the flux polyhedron of the context's construction, by one thread
template <typename G, int KIND>
__device__ __forceinline__ bool poly_scalar(const DevMesh& M, const GeoView<G>& Gv, const GridParam& p,
                                            int j, double Vd, G* vx, G* vy, G* vz, FaceFrame<G>& fr) {
  if constexpr (KIND == VOF_FLUX_EMFPA) return emfpa_scalar<G>(M, Gv, p, j, Vd, vx, vy, vz, fr);
  else if constexpr (KIND == VOF_FLUX_NMFPA) return nmfpa_scalar<G>(M, Gv, p, j, vx, vy, vz, fr);
  else return fmfpa_scalar<G>(M, Gv, p, j, Vd, vx, vy, vz, fr);
}

// Coverage of the flux polyhedron by the candidate cells (Sec. 2.2: at
// CFL <= 1 the donating region lies in the cells around the face). Each
// vertex that is not a node of the face is located in the candidate cells,
// owner and neighbour first, then their node neighbours: in a convex cell
// by its face planes, in a non-convex cell by the winding number of the
// tetrahedra that join its centroid to its fan triangles. A vertex in no
// candidate cell sets kUncovered (the complement form of the mixed path,
// which counts what is not empty as fluid, is then not used); if it lies
// inside the domain's bounding box as well (outside it there is no fluid:
// outflow), kEscaped: the candidate ring does not cover the polyhedron and its
// V_F misses that part (counted, vof_get_stats returns VOF_ECFL).
constexpr unsigned kUncovered = 1u, kEscaped = 2u;

// point (face-local units) in cell k, within tol: a convex cell by its face
// planes (FP32: the cell's plane table), a non-convex cell by the winding
// number of its centroid tetrahedra
template <typename G>
__device__ __noinline__ bool point_in_cell(const DevMesh& M, const GeoView<G>& Gv, const FaceFrame<G>& fr,
                                           int k, G px, G py, G pz, G tol) {
  const int64_t c0 = M.cf_ptr[k], c1 = M.cf_ptr[k + 1];
  if (M.convex[k]) {
    if constexpr (sizeof(G) == 4) {
      const G rx = rel(fr.cx, Gv.ccx[k]), ry = rel(fr.cy, Gv.ccy[k]), rz = rel(fr.cz, Gv.ccz[k]);
      for (int64_t q = c0; q < c1; ++q) {
        const float4 pl = M.cpl32[q];  // inward normal, n.(x - x_k) >= w inside
        if (pl.x * px + pl.y * py + pl.z * pz + (pl.x * rx + pl.y * ry + pl.z * rz - pl.w) * fr.sc < -tol)
          return false;
      }
      return true;
    } else {
      for (int64_t q = c0; q < c1; ++q) {
        const int fs = M.cf[q];
        const int f = fs >= 0 ? fs : ~fs;
        const G sg = fs >= 0 ? G(1) : G(-1);
        const G ox = sg * Gv.fnx[f], oy = sg * Gv.fny[f], oz = sg * Gv.fnz[f];
        // outward distance of p from the face plane, face-local units
        const G d = ox * px + oy * py + oz * pz +
                    (ox * rel(fr.cx, Gv.fcx[f]) + oy * rel(fr.cy, Gv.fcy[f]) + oz * rel(fr.cz, Gv.fcz[f])) * fr.sc;
        if (d > tol) return false;
      }
      return true;
    }
  }
  // winding number of the centroid tetrahedra
  const G rx = rel(Gv.ccx[k], fr.cx) * fr.sc, ry = rel(Gv.ccy[k], fr.cy) * fr.sc,
          rz = rel(Gv.ccz[k], fr.cz) * fr.sc;
  auto det3 = [](G ax, G ay, G az, G bx, G by, G bz, G cx, G cy, G cz) {
    return ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
  };
  int wn = 0;
  for (int64_t q = c0; q < c1; ++q) {
    const int fs = M.cf[q];
    const int f = fs >= 0 ? fs : ~fs;
    const int64_t fb = M.fptr[f];
    const int nI = (int)(M.fptr[f + 1] - fb);
    const int ia = M.fvert[fb];
    const G ax = rel(Gv.vx[ia], fr.cx) * fr.sc - rx, ay = rel(Gv.vy[ia], fr.cy) * fr.sc - ry,
            az = rel(Gv.vz[ia], fr.cz) * fr.sc - rz;
    for (int t = 1; t + 1 < nI; ++t) {
      int ib = M.fvert[fb + t], ic = M.fvert[fb + t + 1];
      if (fs < 0) { const int tmp = ib; ib = ic; ic = tmp; }
      const G bx = rel(Gv.vx[ib], fr.cx) * fr.sc - rx, by = rel(Gv.vy[ib], fr.cy) * fr.sc - ry,
              bz = rel(Gv.vz[ib], fr.cz) * fr.sc - rz;
      const G cx = rel(Gv.vx[ic], fr.cx) * fr.sc - rx, cy = rel(Gv.vy[ic], fr.cy) * fr.sc - ry,
              cz = rel(Gv.vz[ic], fr.cz) * fr.sc - rz;
      const G qx = px - rx, qy = py - ry, qz = pz - rz;
      const G d = det3(ax, ay, az, bx, by, bz, cx, cy, cz);
      if (d == G(0)) continue;
      const G s = d > G(0) ? G(1) : G(-1);
      // p inside the tetrahedron (0, a, b, c): its barycentric weights,
      // each a determinant with p in place of one vertex, all of the sign
      // of d (tolerance in units of the tetrahedron's volume scale)
      const G l1 = s * det3(qx, qy, qz, bx, by, bz, cx, cy, cz);
      const G l2 = s * det3(ax, ay, az, qx, qy, qz, cx, cy, cz);
      const G l3 = s * det3(ax, ay, az, bx, by, bz, qx, qy, qz);
      const G l0 = s * d - l1 - l2 - l3;
      const G tv = tol * s * d;
      if (l0 >= -tv && l1 >= -tv && l2 >= -tv && l3 >= -tv) wn += d > G(0) ? 1 : -1;
    }
  }
  return wn != 0;
}

// p in cell k (one thread): the cell's bounding box first, then an
// axis-aligned box cell is its box, any other cell point_in_cell
template <typename G>
__device__ __forceinline__ bool in_cell(const DevMesh& M, const GeoView<G>& Gv, const FaceFrame<G>& fr,
                                        int k, G px, G py, G pz, G tol) {
  typename Prec<G>::A b[6];
  cell_box<G>(Gv.bb, M.nc, k, b);
  const G lx = rel(b[0], fr.cx) * fr.sc, hx = rel(b[3], fr.cx) * fr.sc;
  if (px < lx - tol || px > hx + tol) return false;
  const G ly = rel(b[1], fr.cy) * fr.sc, hy = rel(b[4], fr.cy) * fr.sc;
  if (py < ly - tol || py > hy + tol) return false;
  const G lz = rel(b[2], fr.cz) * fr.sc, hz = rel(b[5], fr.cz) * fr.sc;
  if (pz < lz - tol || pz > hz + tol) return false;
  return M.convex[k] == 2 || point_in_cell(M, Gv, fr, k, px, py, pz, tol);
}

// coverage bits of the flux polyhedron of face j (one thread; vertices in
// the face-local frame fr). Each vertex to locate (back-traced points and
// apex; EMFPA's side centres are averages of them) is looked up first in
// the cells around the face node it was traced from (the apex: around any
// node of the face), all of them candidate cells, then in the whole
// candidate set (owner, neighbour and their node neighbours); a vertex in no
// candidate cell sets kUncovered, and kEscaped when it lies inside the
// grid's domain box (outside it there is no fluid). A polyhedron whose
// box is flat along an axis has no volume and is not tested.
template <typename G, int KIND>
__device__ __noinline__ unsigned poly_coverage(const DevMesh& M, const GeoView<G>& Gv, const DevState& S,
                                               int j, const G* vx, const G* vy, const G* vz,
                                               const FaceFrame<G>& fr) {
  const G tol = sizeof(G) == 8 ? G(1e-9) : G(2e-5);
  if (!(fr.hi[0] - fr.lo[0] > tol && fr.hi[1] - fr.lo[1] > tol && fr.hi[2] - fr.lo[2] > tol)) return 0u;
  const int I = fr.I, nvb = base_verts<KIND>(I);
  const int64_t fb = M.fptr[j];
  const int own = M.own[j], nbr = M.nbr[j];
  unsigned bits = 0u;
  for (int v = I; v < nvb; ++v) {
    if (KIND == VOF_FLUX_EMFPA && v >= 2 * I && v < 3 * I) continue;  // side centres
    const G px = vx[v], py = vy[v], pz = vz[v];
    bool found = false;
    // the star of the node it was traced from (apex: of any face node): a
    // point within the node's ball lies in one of its cells; else the cells
    // around that node
    const int i0 = v < 2 * I ? v - I : 0, i1 = v < 2 * I ? v - I + 1 : I;
    for (int i = i0; i < i1 && !found; ++i) {
      const G rs = (G)M.rstar[M.fvert[fb + i]] * fr.sc;
      const G dx = px - vx[i], dy = py - vy[i], dz = pz - vz[i];
      found = dx * dx + dy * dy + dz * dz < rs * rs;
    }
    for (int i = i0; i < i1 && !found; ++i) {
      const int node = M.fvert[fb + i];
      for (int64_t q = M.vc_ptr[node]; q < M.vc_ptr[node + 1] && !found; ++q)
        found = in_cell(M, Gv, fr, M.vc[q], px, py, pz, tol);
    }
    // the whole candidate set
    for (int pass = 0; pass < 2 && !found; ++pass) {
      const int c0 = pass == 0 ? own : nbr;
      if (c0 < 0) break;
      found = in_cell(M, Gv, fr, c0, px, py, pz, tol);
      for (int64_t q = M.nb_ptr[c0]; q < M.nb_ptr[c0 + 1] && !found; ++q)
        found = in_cell(M, Gv, fr, M.nb[q], px, py, pz, tol);
    }
    if (found) continue;
    bits |= kUncovered;
    const int g = M.n_grids == 1 ? 0 : grid_of(M.face_off, M.n_grids, j);
    const double* b = S.dombox + 6 * g;
    const double L = (double)fr.L;
    const double ax = absd(fr.cx) + L * (double)px, ay = absd(fr.cy) + L * (double)py,
                 az = absd(fr.cz) + L * (double)pz;
    const double eps = 1e-9 * L;
    if (ax > b[0] + eps && ax < b[3] - eps && ay > b[1] + eps && ay < b[4] - eps && az > b[2] + eps &&
        az < b[5] - eps)
      bits |= kEscaped;
  }
  return bits;
}

// the polyhedron of face j into shared memory by lane 0 (the other lanes
// wait): the flux kernel's fallback beyond the prebuilt capacity and the
// polyhedron export
template <typename G, int KIND, int GW>
__device__ __noinline__ bool build_polyhedron(const DevMesh& M, const GeoView<G>& Gv, const GridParam& p,
                                              int j, double Vd, Poly<G, GW>& P, FaceFrame<G>& frs, int lane) {
  int ok = 0;
  if (lane == 0) ok = poly_scalar<G, KIND>(M, Gv, p, j, Vd, P.bx, P.by, P.bz, frs) ? 1 : 0;
  ok = gshfl<GW>(ok, 0);
  gsync<GW>();
  return ok != 0;
}

// the polyhedron of active face w built by lane 0 (past the prebuilt
// capacity), with its coverage bits written as k_prebuild writes them
template <typename G, int KIND, int GW>
__device__ __noinline__ bool build_polyhedron_cov(const DevMesh& M, const GeoView<G>& Gv, const DevState& S,
                                                  const GridParam& p, int j, unsigned w, double Vd,
                                                  Poly<G, GW>& P, FaceFrame<G>& frs, int lane) {
  int ok = 0;
  if (lane == 0) {
    ok = poly_scalar<G, KIND>(M, Gv, p, j, Vd, P.bx, P.by, P.bz, frs) ? 1 : 0;
    const unsigned cov = ok ? poly_coverage<G, KIND>(M, Gv, S, j, P.bx, P.by, P.bz, frs) : 0u;
    S.cover8[w] = (uint8_t)cov;
    if (cov & kEscaped) atomicAdd(S.cnt + kNEscape, 1ull);
  }
  ok = gshfl<GW>(ok, 0);
  gsync<GW>();
  return ok != 0;
}

__device__ __forceinline__ bool sorted_contains(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == key;
}

// vol(P ∩ K ∩ X) in face-local units, K the convex region of the np
// half-spaces P.pl[0..np) (inner side a.x + b >= 0) and X either all space
// (plic = false) or the half-space P.pl[NF] (the PLIC plane, oriented to
// the side that is wanted).
// The planes are first tested against the base polyhedron's vertices (one
// ballot per plane): a plane with every vertex outside empties the
// intersection, a plane with none outside is skipped, and only the planes
// that cut are clipped: all but the last topologically, the last one inside
// the volume sum. *whole = 1 when P lies inside K ∩ X (the result is then
// the volume of P itself). Vertices within tol of a plane count as on its
// inner side; tol is a few ulps of the face-local unit, so the volume this
// neglects is of the order of the rounding of the plane itself.
template <typename G, int KIND, int GW>
__device__ GVOF_PLANES_ATTR G truncate_planes(Poly<G, GW>& P, int np, bool has_plic, const FaceFrame<G>& fr,
                                          G Vl, int lane, unsigned& err, int* whole) {
  constexpr int NF = Poly<G, GW>::NF;
  const G tol = sizeof(G) == 8 ? G(1e-14) : G(2e-7);
  *whole = 0;
  const bool hv = lane < base_verts<KIND>(fr.I);
  const G bx = hv ? P.bx[lane] : G(0), by = hv ? P.by[lane] : G(0), bz = hv ? P.bz[lane] : G(0);
  unsigned cut = 0u;
  for (int g = 0; g < np; ++g) {
    const G ph = P.pl[g][0] * bx + P.pl[g][1] * by + P.pl[g][2] * bz + P.pl[g][3];
    const unsigned out = gballot<GW>(hv && ph < -tol);
    const unsigned in = gballot<GW>(hv && ph > tol);
    if (in == 0u && out != 0u) return G(0);  // P on the outer side of a plane
    if (out) cut |= 1u << g;
  }
  bool plic = false;
  if (has_plic) {
    const G ph = P.pl[NF][0] * bx + P.pl[NF][1] * by + P.pl[NF][2] * bz + P.pl[NF][3];
    const unsigned out = gballot<GW>(hv && ph < -tol);
    const unsigned in = gballot<GW>(hv && ph > tol);
    if (in == 0u && out != 0u) return G(0);  // P on the other side of the interface
    plic = out != 0u;
  }
  if (cut == 0u && !plic) { *whole = 1; return Vl; }  // P inside K ∩ X
  int last;
  if (plic) {
    last = NF;
  } else {
    last = 31 - __clz(cut);
    cut &= ~(1u << last);
  }
  PolyState st;
  restore_base<G, KIND>(P, st, fr.I, fr.split, lane);
  int res = 0;
  while (cut && res != 2) {
    const int g = __ffs(cut) - 1;
    cut &= cut - 1u;
    res = clip(P, st, P.pl[g][0], P.pl[g][1], P.pl[g][2], P.pl[g][3], lane, err);
  }
  if (res == 2) return G(0);
  if (sizeof(G) == 8) {
    // FP64: the streaming cut recomputes every cut point twice, and FP64
    // divisions are costly on this GPU; clip topologically instead
    res = clip(P, st, P.pl[last][0], P.pl[last][1], P.pl[last][2], P.pl[last][3], lane, err);
    return res == 2 ? G(0) : volume(P, st, lane);
  }
  return volume_cut(P, st, P.pl[last][0], P.pl[last][1], P.pl[last][2], P.pl[last][3], lane);
}

// vol(P ∩ K ∩ X) for a non-convex cell K: signed sum over the tetrahedra
// that join its centroid to the fan triangles of its faces (winding-number
// decomposition, valid for any closed cell); the PLIC half-space, if any, is
// already in P.pl[NF]
template <typename G, int KIND, int GW>
__device__ __noinline__ G truncate_nonconvex(const DevMesh& M, const GeoView<G>& Gv, int k,
                                             int64_t c0, int nfk, bool tag0, const FaceFrame<G>& fr,
                                             G Vl, Poly<G, GW>& P, int lane, unsigned& err) {
  // one lane per face of the cell: a half-warp group takes cells of at most
  // 16 faces (the flux kernel uses it only on such grids)
  if (nfk > GW) { err |= 1u; return G(0); }
  const G rx = rel(Gv.ccx[k], fr.cx) * fr.sc, ry = rel(Gv.ccy[k], fr.cy) * fr.sc,
          rz = rel(Gv.ccz[k], fr.cz) * fr.sc;
  // fan triangles per face, and their running count (lanes over faces)
  int ntri = 0, fs_l = 0;
  int64_t fb_l = 0;
  if (lane < nfk) {
    fs_l = M.cf[c0 + lane];
    const int f = fs_l >= 0 ? fs_l : ~fs_l;
    fb_l = M.fptr[f];
    ntri = (int)(M.fptr[f + 1] - fb_l) - 2;
  }
  int incl = ntri;
  for (int d = 1; d < GW; d <<= 1) {
    const int t = gshfl_up<GW>(incl, d);
    if (lane >= d) incl += t;
  }
  const int total = gshfl<GW>(incl, GW - 1);
  const int first = incl - ntri;
  G v = G(0);
  // lanes over tetrahedra, GW at a time: build, orient, reject by bounding box
  for (int base = 0; base < total; base += GW) {
    const int id = base + lane;
    G T[4][3];
    G sgn = G(0);
    bool keep = false;
    // face holding tetrahedron id: the last face whose first <= id
    int q = 0;
    for (int r = 0; r < nfk; ++r) {
      const int fr_first = gshfl<GW>(first, r);
      if (fr_first <= id) q = r;
    }
    const int fs = gshfl<GW>(fs_l, q & (GW - 1));
    const int64_t fb = gshfl<GW>(fb_l, q & (GW - 1));
    const int fq_first = gshfl<GW>(first, q & (GW - 1));
    if (id < total) {
      const int t = id - fq_first + 1;
      int ia = M.fvert[fb], ib = M.fvert[fb + t], ic = M.fvert[fb + t + 1];
      if (fs < 0) { const int tmp = ib; ib = ic; ic = tmp; }
      T[0][0] = rx; T[0][1] = ry; T[0][2] = rz;
      const int ids[3] = {ia, ib, ic};
      for (int e = 0; e < 3; ++e) {
        T[e + 1][0] = rel(Gv.vx[ids[e]], fr.cx) * fr.sc;
        T[e + 1][1] = rel(Gv.vy[ids[e]], fr.cy) * fr.sc;
        T[e + 1][2] = rel(Gv.vz[ids[e]], fr.cz) * fr.sc;
      }
      const G ux = T[1][0] - T[0][0], uy = T[1][1] - T[0][1], uz = T[1][2] - T[0][2];
      const G wx = T[2][0] - T[0][0], wy = T[2][1] - T[0][1], wz = T[2][2] - T[0][2];
      const G zx = T[3][0] - T[0][0], zy = T[3][1] - T[0][1], zz = T[3][2] - T[0][2];
      const G det = ux * (wy * zz - wz * zy) + uy * (wz * zx - wx * zz) + uz * (wx * zy - wy * zx);
      sgn = det > G(0) ? G(1) : G(-1);
      G lo0 = T[0][0], hi0 = T[0][0], lo1 = T[0][1], hi1 = T[0][1], lo2 = T[0][2], hi2 = T[0][2];
      for (int e = 1; e < 4; ++e) {
        lo0 = min(lo0, T[e][0]); hi0 = max(hi0, T[e][0]);
        lo1 = min(lo1, T[e][1]); hi1 = max(hi1, T[e][1]);
        lo2 = min(lo2, T[e][2]); hi2 = max(hi2, T[e][2]);
      }
      keep = det != G(0) && fr.hi[0] > lo0 && fr.lo[0] < hi0 && fr.hi[1] > lo1 &&
             fr.lo[1] < hi1 && fr.hi[2] > lo2 && fr.lo[2] < hi2;
    }
    unsigned bal = gballot<GW>(keep);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1u;
      G Tq[4][3];
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) Tq[a][d] = gshfl<GW>(T[a][d], src);
      const G sg = gshfl<GW>(sgn, src);
      // inward planes of the tetrahedron: face opposite vertex a, outward
      // normal (q1 - q0) x (q2 - q0) for a positive tetrahedron
      if (lane < 4) {
        const int o0 = lane == 0 ? 1 : 0;
        const int o1 = lane == 0 ? 2 : (lane == 1 ? 3 : (lane == 2 ? 1 : 2));
        const int o2 = lane == 0 ? 3 : (lane == 1 ? 2 : (lane == 2 ? 3 : 1));
        const G ax = Tq[o1][0] - Tq[o0][0], ay = Tq[o1][1] - Tq[o0][1], az = Tq[o1][2] - Tq[o0][2];
        const G cx = Tq[o2][0] - Tq[o0][0], cy = Tq[o2][1] - Tq[o0][1], cz = Tq[o2][2] - Tq[o0][2];
        G nx = (ay * cz - az * cy) * sg, ny = (az * cx - ax * cz) * sg, nz = (ax * cy - ay * cx) * sg;
        const G nn = G(1) / sqrt(nx * nx + ny * ny + nz * nz);
        nx *= nn; ny *= nn; nz *= nn;
        P.pl[lane][0] = -nx; P.pl[lane][1] = -ny; P.pl[lane][2] = -nz;
        P.pl[lane][3] = nx * Tq[o0][0] + ny * Tq[o0][1] + nz * Tq[o0][2];
      }
      gsync<GW>();
      int w = 0;
      v += sg * truncate_planes<G, KIND>(P, 4, tag0, fr, Vl, lane, err, &w);
    }
  }
  return v;
}

// vol(P ∩ cell k ∩ X_k) in face-local units, X_k the fluid of cell k
// (empty_side = false: all of a full cell, the PLIC half-space of an
// interfacial cell) or its empty part (empty_side = true: all of an empty
// cell, the complementary half-space of an interfacial cell). A convex cell
// is the intersection of its face half-spaces; a non-convex cell is the
// signed sum of the tetrahedra that join its centroid to the fan triangles of
// its faces (winding-number decomposition, valid for any closed cell).
template <typename G, int KIND, int GW>
__device__ GVOF_CELL_ATTR G truncate_in_cell(const DevMesh& M, const GeoView<G>& Gv,
                                           const DevState& S, int k, const FaceFrame<G>& fr, G Vl,
                                           Poly<G, GW>& P, int lane, unsigned& err, bool empty_side,
                                           int* whole) {
  constexpr int NF = Poly<G, GW>::NF;
  *whole = 0;
  const int8_t tk = S.tc[k];
  if (tk == (empty_side ? 1 : -1)) return G(0);
  const bool tag0 = tk == 0;
  if (tag0 && lane == 0) {
    // half-space of the PLIC plane on the wanted side: n.(x - x_k) + C >= 0
    G pn0 = Gv.pnx[k], pn1 = Gv.pny[k], pn2 = Gv.pnz[k];
    G pnb = (pn0 * rel(fr.cx, Gv.ccx[k]) + pn1 * rel(fr.cy, Gv.ccy[k]) + pn2 * rel(fr.cz, Gv.ccz[k]) +
             Gv.pC[k]) * fr.sc;
    if (empty_side) { pn0 = -pn0; pn1 = -pn1; pn2 = -pn2; pnb = -pnb; }
    P.pl[NF][0] = pn0; P.pl[NF][1] = pn1; P.pl[NF][2] = pn2; P.pl[NF][3] = pnb;
  }
  const int64_t c0 = M.cf_ptr[k];
  const int nfk = (int)(M.cf_ptr[k + 1] - c0);
  if (M.convex[k]) {
    // inward half-spaces of cell k: -n_out.(x - p_g) >= 0, i.e. in the local
    // frame a = -n_out, b = -n_out.(c - p_g) / L
    if constexpr (sizeof(G) == 4) {
      // FP32: from the cell's plane table, n.(x - x_k) >= d in the face-local frame
      if (lane < nfk) {
        const G rx = rel(fr.cx, Gv.ccx[k]), ry = rel(fr.cy, Gv.ccy[k]), rz = rel(fr.cz, Gv.ccz[k]);
        const float4 q = M.cpl32[c0 + lane];
        P.pl[lane][0] = q.x; P.pl[lane][1] = q.y; P.pl[lane][2] = q.z;
        P.pl[lane][3] = (q.x * rx + q.y * ry + q.z * rz - q.w) * fr.sc;
      }
    } else if (lane < nfk) {
      const int fs = M.cf[c0 + lane];
      const int f = fs >= 0 ? fs : ~fs;
      const G sg = fs >= 0 ? G(1) : G(-1);
      const G ox = sg * Gv.fnx[f], oy = sg * Gv.fny[f], oz = sg * Gv.fnz[f];
      P.pl[lane][0] = -ox; P.pl[lane][1] = -oy; P.pl[lane][2] = -oz;
      P.pl[lane][3] = -(ox * rel(fr.cx, Gv.fcx[f]) + oy * rel(fr.cy, Gv.fcy[f]) +
                        oz * rel(fr.cz, Gv.fcz[f])) * fr.sc;
    }
    gsync<GW>();
    return truncate_planes<G, KIND>(P, nfk, tag0, fr, Vl, lane, err, whole);
  }
  return truncate_nonconvex<G, KIND>(M, Gv, k, c0, nfk, tag0, fr, Vl, P, lane, err);
}

// the filters of a candidate cell k: the local bounding box of the
// polyhedron, then (FP32, convex cells other than axis-aligned boxes, whose
// box test is already this one) the cell's face planes: a cell with a plane
// that has every base vertex (bx, by, bz) strictly outside cannot meet P.
// The flux kernel and the prebuild thread call this one function, so both
// take the same decisions.
template <typename G, int KIND>
__device__ __forceinline__ bool cell_may_meet(const DevMesh& M, const GeoView<G>& Gv,
                                              const FaceFrame<G>& fr, const G* bx, const G* by,
                                              const G* bz, int k) {
  typename Prec<G>::A b[6];
  cell_box<G>(Gv.bb, M.nc, k, b);
  const G lx = rel(b[0], fr.cx) * fr.sc, hx = rel(b[3], fr.cx) * fr.sc;
  const G ly = rel(b[1], fr.cy) * fr.sc, hy = rel(b[4], fr.cy) * fr.sc;
  const G lz = rel(b[2], fr.cz) * fr.sc, hz = rel(b[5], fr.cz) * fr.sc;
  if (!(fr.hi[0] > lx && fr.lo[0] < hx && fr.hi[1] > ly && fr.lo[1] < hy && fr.hi[2] > lz &&
        fr.lo[2] < hz))
    return false;
  if constexpr (sizeof(G) == 4) {
    if (M.convex[k] == 1) {
      const int64_t q0 = M.cf_ptr[k];
      const int nfk = (int)(M.cf_ptr[k + 1] - q0);
      const int nvb = base_verts<KIND>(fr.I);
      const G rx = rel(fr.cx, Gv.ccx[k]), ry = rel(fr.cy, Gv.ccy[k]), rz = rel(fr.cz, Gv.ccz[k]);
      for (int g = 0; g < nfk; ++g) {
        const float4 q = M.cpl32[q0 + g];
        const G b = (q.x * rx + q.y * ry + q.z * rz - q.w) * fr.sc;
        bool out = true;
        for (int v = 0; v < nvb && out; ++v) out = q.x * bx[v] + q.y * by[v] + q.z * bz[v] + b < G(-2e-7);
        if (out) return false;
      }
    }
  }
  return true;
}

// candidate idx of one pass over face j's candidate cells (pass 0: the
// owner's node neighbours and the owner; pass 1: the neighbour's and the
// neighbour, minus those already seen), filtered by cell_may_meet with the
// base vertices (bx, by, bz); returns the cell (-1: none) and its tag
template <typename G, int KIND>
__device__ __forceinline__ int candidate_at(const DevMesh& M, const GeoView<G>& Gv, const DevState& S,
                                            const FaceFrame<G>& fr, const G* bx, const G* by,
                                            const G* bz, int own, int64_t a0, int na, int pass, int c0,
                                            int64_t b0, int nb, int idx, int8_t& tk) {
  int k = -1;
  if (idx < nb) k = (idx == nb - 1) ? c0 : M.nb[b0 + idx];
  if (k >= 0 && pass == 1 && (k == own || sorted_contains(M.nb + a0, na, k))) k = -1;
  tk = 0;
  if (k >= 0 && !cell_may_meet<G, KIND>(M, Gv, fr, bx, by, bz, k)) k = -1;
  if (k >= 0) tk = S.tc[k];
  return k;
}

template <typename G, int KIND, int GW>
__device__ __forceinline__ int candidate(const DevMesh& M, const GeoView<G>& Gv, const DevState& S,
                                         const FaceFrame<G>& fr, const Poly<G, GW>& P, int own, int64_t a0,
                                         int na, int pass, int c0, int64_t b0, int nb, int idx,
                                         int8_t& tk) {
  return candidate_at<G, KIND>(M, Gv, S, fr, P.bx, P.by, P.bz, own, a0, na, pass, c0, b0, nb, idx, tk);
}

// V_F of face j in face-local units (Sec. 2.2): the candidate cells (owner,
// its node neighbours, then the neighbour and its node neighbours not seen
// yet: donating regions of several cells) met by the bounding box of P are
// listed first, with their tags. The fluid form sums vol(P ∩ cell ∩ fluid)
// over the full and interfacial cells. The complement form (FP32 only, an
// interior face, where P lies in the candidate cells at CFL <= 1 so that
// fluid + empty = V_d) gives V_d minus the sum of the empty parts over the
// interfacial and empty cells, so that the FP32 error scales with the empty
// part. The form is chosen from the tags so that a polyhedron that lies
// only in fluid gives exactly V_d and one that lies only in empty space
// exactly 0: complement when no empty cell is met, fluid when no full cell
// is, otherwise by the donating cell's F. Returns V_F / L^3; *whole: P lies
// in the fluid (1) or empty (2) part of one cell (V_F = V_d or 0 exactly).
// cover: the coverage bits of P (poly_coverage); the complement form needs a
// covered P.
template <typename G, int KIND, int GW>
__device__ GVOF_OUTER_ATTR G sweep_candidates(const DevMesh& M, const GeoView<G>& Gv, const DevState& S, int j,
                              const FaceFrame<G>& fr, double Vd, G Vl, Poly<G, GW>& P, int lane,
                              unsigned& err, int* whole, bool* complement, unsigned cover,
                              unsigned long long& n_trunc, unsigned w) {
  const int own = M.own[j], nbr = M.nbr[j];
  const int64_t a0 = M.nb_ptr[own];
  const int na = (int)(M.nb_ptr[own + 1] - a0);
  constexpr int cap = cand_cap<G>();
  int n = cap + 1;  // FP64: the fluid form, no list (the cells are scanned once)
  bool neg = false, pos = false;
  bool listed = false;
  if constexpr (sizeof(G) == 4) {
    n = 0;
    // the list built with the polyhedron, when it fits
    if (S.fm_cand != nullptr && (int64_t)w < S.fm_cap) {
      const unsigned info = S.fm_cinfo[w];
      const int cnt = (int)(info & 63u);
      if (cnt <= kPreCand) {
        listed = true;
        n = cnt;
        neg = ((info >> 6) & 1u) != 0u;
        pos = ((info >> 7) & 1u) != 0u;
        for (int i = lane; i < cnt; i += GW) P.cand[i] = S.fm_cand[(size_t)w * kPreCand + i];
      }
    }
  }
  for (int pass = 0; sizeof(G) == 4 && !listed && pass < 2; ++pass) {
    const int c0 = pass == 0 ? own : nbr;
    if (c0 < 0) break;
    const int64_t b0 = M.nb_ptr[c0];
    const int nb = (int)(M.nb_ptr[c0 + 1] - b0) + 1;
    for (int base = 0; base < nb; base += GW) {
      int8_t tk;
      const int k = candidate<G, KIND>(M, Gv, S, fr, P, own, a0, na, pass, c0, b0, nb, base + lane, tk);
      const unsigned bal = gballot<GW>(k >= 0);
      if (gany<GW>(k >= 0 && tk == -1)) neg = true;
      if (gany<GW>(k >= 0 && tk == 1)) pos = true;
      const int at = n + __popc(bal & ((1u << lane) - 1u));
      if (k >= 0 && at < cap) P.cand[at] = k;
      n += __popc(bal);
    }
  }
  gsync<GW>();
  bool comp = false;
  if (sizeof(G) == 4 && nbr >= 0 && !(cover & kUncovered)) {
    if (!neg && pos) comp = true;
    else if (neg && !pos) comp = false;
    else comp = S.F[Vd > 0.0 ? own : nbr] > 0.5;
  }
  *complement = comp;
  *whole = 0;
  // the cells the form needs: fluid form tags 1 and 0, complement 0 and -1
  const int8_t skip = comp ? 1 : -1;
  G v = G(0);
  if (n <= cap) {
    for (int i = 0; i < n; ++i) {
      const int kk = P.cand[i];
      if (S.tc[kk] == skip) continue;
      int w = 0;
      v += truncate_in_cell<G, KIND>(M, Gv, S, kk, fr, Vl, P, lane, err, comp, &w);
      ++n_trunc;
      if (w) { *whole = comp ? 2 : 1; return G(0); }  // no other cell meets P
    }
    return v;
  }
  // more candidates than the list holds: the same cells, scanned again
  for (int pass = 0; pass < 2; ++pass) {
    const int c0 = pass == 0 ? own : nbr;
    if (c0 < 0) break;
    const int64_t b0 = M.nb_ptr[c0];
    const int nb = (int)(M.nb_ptr[c0 + 1] - b0) + 1;
    for (int base = 0; base < nb; base += GW) {
      int8_t tk;
      const int k = candidate<G, KIND>(M, Gv, S, fr, P, own, a0, na, pass, c0, b0, nb, base + lane, tk);
      unsigned bal = gballot<GW>(k >= 0 && tk != skip);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1u;
        const int kk = gshfl<GW>(k, src);
        int w = 0;
        v += truncate_in_cell<G, KIND>(M, Gv, S, kk, fr, Vl, P, lane, err, comp, &w);
        ++n_trunc;
        if (w) { *whole = comp ? 2 : 1; return G(0); }
      }
    }
  }
  return v;
}

// flux polyhedra of the first fm_cap active faces, one thread per face
// (poly_scalar), into the prebuilt buffer the flux kernel reads
template <typename G, int KIND>
__global__ void __launch_bounds__(128) k_prebuild(DevMesh M, GeoView<G> Gv, DevState S) {
  const unsigned n_af = (unsigned)S.cnt[kNAfaces];
  const unsigned nb = (unsigned)min((int64_t)n_af, S.fm_cap);
  G* fv = (G*)S.fm_v;
  G* ff = (G*)S.fm_f;
  for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < nb; w += gridDim.x * blockDim.x) {
    const int j = S.afaces[w];
    const GridParam& gp = S.gp[M.n_grids == 1 ? 0 : grid_of(M.face_off, M.n_grids, j)];
    if (gp.gdt == 0.0) {
      // a grid that does not move this step (a batch slot whose request is
      // done): the flux kernel gives its faces V_F = 0 without a polyhedron
      S.fm_meta[w] = 0u;
      S.cover8[w] = 0;
      continue;
    }
    const double Vd = S.srate[j] * gp.gdt;
    G vx[kFmSlots], vy[kFmSlots], vz[kFmSlots];
    FaceFrame<G> fr;
    const bool ok = poly_scalar<G, KIND>(M, Gv, gp, j, Vd, vx, vy, vz, fr);
    S.fm_meta[w] = (uint32_t)fr.I | ((uint32_t)fr.degenerate << 8) | ((uint32_t)fr.edgeon << 16) |
                   ((uint32_t)(ok ? 1 : 0) << 24);
    const unsigned cov = ok ? poly_coverage<G, KIND>(M, Gv, S, j, vx, vy, vz, fr) : 0u;
    S.cover8[w] = (uint8_t)cov;
    if (cov & kEscaped) atomicAdd(S.cnt + kNEscape, 1ull);
    if (!ok) continue;

    S.fm_split[w] = fr.split;
    G* f = ff + (size_t)w * 7;
    f[0] = fr.L;
    f[1] = fr.lo[0]; f[2] = fr.lo[1]; f[3] = fr.lo[2];
    f[4] = fr.hi[0]; f[5] = fr.hi[1]; f[6] = fr.hi[2];
    G* v = fv + (size_t)w * kFmSlots * 3;
    for (int q = 0; q < base_verts<KIND>(fr.I); ++q) {
      v[3 * q] = vx[q]; v[3 * q + 1] = vy[q]; v[3 * q + 2] = vz[q];
    }
  }
}

// the candidate lists of the prebuilt polyhedra (FP32 path), 16 lanes per
// face: the search the flux kernel's sweep_candidates would make, with the
// same filter (candidate_at), in the same order, with the census of the
// tags. Each lane takes two cells of a pass at once so that their gathers
// are in flight together, and the groups hold little state, so that many of
// them hide the gathers' latency. The neighbour's pass drops the cells the
// owner's pass accepted (a cell of both rings passes the same filter in
// both, so this is the flux kernel's de-duplication). A face whose list
// exceeds kPreCand is left to the flux kernel's own search.
constexpr int kListWarps = 8;
constexpr int kListGroups = 2 * kListWarps;
template <typename G, int KIND>
__global__ void __launch_bounds__(kListWarps * 32) k_candlist(DevMesh M, GeoView<G> Gv, DevState S) {
  __shared__ G bv[kListGroups][3][kFmSlots];
  __shared__ int32_t seen[kListGroups][kPreCand];
  const int lane = threadIdx.x & 15, grp = threadIdx.x >> 4;
  const unsigned sh = threadIdx.x & 16u;
  const unsigned gm = 0xffffu << sh;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned n_af = (unsigned)S.cnt[kNAfaces];
  const unsigned nw = (unsigned)min((int64_t)n_af, S.fm_cap);
  G* bx = bv[grp][0];
  G* by = bv[grp][1];
  G* bz = bv[grp][2];
  int32_t* sn = seen[grp];
  for (unsigned w = blockIdx.x * kListGroups + grp; w < nw; w += gridDim.x * kListGroups) {
    const uint32_t meta = S.fm_meta[w];
    if (!((meta >> 24) & 1u)) continue;  // no polyhedron: the flux kernel skips the face
    const int j = S.afaces[w];
    FaceFrame<G> fr;
    fr.I = (int)(meta & 255u);
    const G* f = (const G*)S.fm_f + (size_t)w * 7;
    fr.cx = Gv.fcx[j]; fr.cy = Gv.fcy[j]; fr.cz = Gv.fcz[j];
    fr.L = f[0];
    fr.sc = G(1) / fr.L;
    fr.lo[0] = f[1]; fr.lo[1] = f[2]; fr.lo[2] = f[3];
    fr.hi[0] = f[4]; fr.hi[1] = f[5]; fr.hi[2] = f[6];
    for (int v = lane; v < base_verts<KIND>(fr.I); v += 16) {
      const G* p = (const G*)S.fm_v + ((size_t)w * kFmSlots + v) * 3;
      bx[v] = p[0]; by[v] = p[1]; bz[v] = p[2];
    }
    __syncwarp(gm);
    const int own = M.own[j], nbr = M.nbr[j];
    int n = 0, n0 = 0;
    bool neg = false, pos = false;
    int32_t* out = S.fm_cand + (size_t)w * kPreCand;
    for (int pass = 0; pass < 2; ++pass) {
      const int c0 = pass == 0 ? own : nbr;
      if (c0 < 0) break;
      const int64_t b0 = M.nb_ptr[c0];
      const int nb = (int)(M.nb_ptr[c0 + 1] - b0) + 1;
      const int m0 = n0 < kPreCand ? n0 : kPreCand;
      for (int base = 0; base < nb; base += 32) {
        int8_t t0, t1;
        // pass 0 semantics of candidate_at: the filter alone (no de-duplication)
        int k0 = candidate_at<G, KIND>(M, Gv, S, fr, bx, by, bz, own, 0, 0, 0, c0, b0, nb, base + lane, t0);
        int k1 = candidate_at<G, KIND>(M, Gv, S, fr, bx, by, bz, own, 0, 0, 0, c0, b0, nb, base + 16 + lane,
                                       t1);
        if (pass == 1) {
          for (int i = 0; i < m0 && (k0 >= 0 || k1 >= 0); ++i) {
            const int q = sn[i];
            if (q == k0) k0 = -1;
            if (q == k1) k1 = -1;
          }
        }
        const unsigned b0m = (__ballot_sync(gm, k0 >= 0) >> sh) & 0xffffu;
        const unsigned b1m = (__ballot_sync(gm, k1 >= 0) >> sh) & 0xffffu;
        if (__any_sync(gm, (k0 >= 0 && t0 == -1) || (k1 >= 0 && t1 == -1))) neg = true;
        if (__any_sync(gm, (k0 >= 0 && t0 == 1) || (k1 >= 0 && t1 == 1))) pos = true;
        const int at0 = n + __popc(b0m & lt);
        if (k0 >= 0 && at0 < kPreCand) {
          out[at0] = k0;
          if (pass == 0) sn[at0] = k0;
        }
        n += __popc(b0m);
        const int at1 = n + __popc(b1m & lt);
        if (k1 >= 0 && at1 < kPreCand) {
          out[at1] = k1;
          if (pass == 0) sn[at1] = k1;
        }
        n += __popc(b1m);
      }
      if (pass == 0) n0 = n;
      __syncwarp(gm);
    }
    if (lane == 0) S.fm_cinfo[w] = (uint8_t)((n <= kPreCand ? n : 63) | (neg ? 64 : 0) | (pos ? 128 : 0));
    __syncwarp(gm);
  }
}

// the flux polyhedron of active face w: prebuilt below fm_cap, else built
// here by lane 0 with the same arithmetic
template <typename G, int KIND, int GW>
__device__ bool poly_for_face(const DevMesh& M, const GeoView<G>& Gv, const DevState& S, unsigned w,
                              int j, const GridParam& p, double Vd, Poly<G, GW>& P, FaceFrame<G>& fr,
                              int lane) {
  if ((int64_t)w >= S.fm_cap) return build_polyhedron_cov<G, KIND>(M, Gv, S, p, j, w, Vd, P, fr, lane);
  const uint32_t meta = S.fm_meta[w];
  const int I = (int)(meta & 255u);
  const bool ok = (meta >> 24) & 1u;
  if (lane == 0) {
    fr.I = I;
    fr.degenerate = (int)((meta >> 8) & 255u);
    fr.edgeon = (int)((meta >> 16) & 255u);
    if (ok) {
      const G* f = (const G*)S.fm_f + (size_t)w * 7;
      fr.cx = Gv.fcx[j]; fr.cy = Gv.fcy[j]; fr.cz = Gv.fcz[j];
      fr.L = f[0];
      fr.sc = G(1) / fr.L;
      fr.lo[0] = f[1]; fr.lo[1] = f[2]; fr.lo[2] = f[3];
      fr.hi[0] = f[4]; fr.hi[1] = f[5]; fr.hi[2] = f[6];
      fr.split = S.fm_split[w];
    }
  }
  if (ok && lane < base_verts<KIND>(I)) {
    const G* v = (const G*)S.fm_v + ((size_t)w * kFmSlots + lane) * 3;
    P.bx[lane] = v[0]; P.by[lane] = v[1]; P.bz[lane] = v[2];
  }
  gsync<GW>();
  return ok;
}

// the next active face for this lane group: faces are dealt one at a time
// from a counter, so a group that drew cheap faces takes more and none idles
// while another still holds a queue (the results do not depend on the order)
template <int GW>
__device__ __forceinline__ unsigned next_face(const DevState& S, int lane) {
  unsigned w = 0u;
  if (lane == 0) w = (unsigned)atomicAdd(S.cnt + kFluxNext, 1ull);
  return gshfl<GW>(w, 0);
}

static_assert(sizeof(GridParam) % sizeof(double) == 0 && sizeof(GridParam) / sizeof(double) <= 16,
              "a half warp stages the grid parameters");

// one lane group (a warp, GW = 32, or a half warp, GW = 16) per active face
template <typename G, int KIND, int GW>
__global__ void __launch_bounds__(kWarps * 32, GVOF_FLUX_MINB) k_flux(DevMesh M, GeoView<G> Gv, DevState S) {
  constexpr int kGroups = kWarps * 32 / GW;
  __shared__ Poly<G, GW> polys[kGroups];
  __shared__ GridParam wgp[kGroups];
  __shared__ FaceFrame<G> wfr[kGroups];
  const int lane = threadIdx.x & (GW - 1), wib = threadIdx.x / GW;
  Poly<G, GW>& P = polys[wib];
  FaceFrame<G>& fr = wfr[wib];
  const unsigned n_af = (unsigned)S.cnt[kNAfaces];
  unsigned long long n_trunc = 0, n_over = 0, n_deg = 0, n_edge = 0;
  for (unsigned w = next_face<GW>(S, lane); w < n_af; w = next_face<GW>(S, lane)) {
    const int j = S.afaces[w];
    // the face's grid parameters, staged in shared memory (read at use)
    {
      const int gi = M.n_grids == 1 ? 0 : grid_of(M.face_off, M.n_grids, j);
      constexpr int nw = (int)(sizeof(GridParam) / sizeof(double));
      if (lane < nw) ((double*)&wgp[wib])[lane] = ((const double*)&S.gp[gi])[lane];
      gsync<GW>();
    }
    if (wgp[wib].gdt == 0.0) {
      // no displacement this step (g dt = 0: a batch slot that does not
      // move): every back-traced point is its face point, so the flux
      // polyhedron is the face itself and V_F = 0 exactly
      if (lane == 0) {
        S.VF[j] = 0.0;
        if constexpr (sizeof(G) == 4) S.fexact[j] = 1;
      }
      continue;
    }
    const double Vd = S.srate[j] * wgp[wib].gdt;  // V_d of Eq. a-donacion
    if (!poly_for_face<G, KIND>(M, Gv, S, w, j, wgp[wib], Vd, P, fr, lane)) {
      if (lane == 0) {
        S.VF[j] = 0.0;
        if constexpr (sizeof(G) == 4) S.fexact[j] = 0;
      }
      ++n_over;
      continue;
    }
    n_deg += fr.degenerate;
    n_edge += fr.edgeon;
    unsigned err = 0u;
    const G Vl = (G)Vd * (fr.sc * fr.sc * fr.sc);  // volume of P, local units
    const G L3 = fr.L * fr.L * fr.L;
    int wh = 0;
    bool comp = false;
    const G v = sweep_candidates<G, KIND>(M, Gv, S, j, fr, Vd, Vl, P, lane, err, &wh, &comp,
                                          (unsigned)S.cover8[w], n_trunc, w);
    double VFj;
    if (wh == 1) VFj = Vd;  // P inside the fluid of one cell: exactly V_d
    else if (wh == 2) VFj = 0.0;  // P inside the empty part of one cell
    else VFj = comp ? Vd - (double)(v * L3) : (double)(v * L3);
    if (err) ++n_over;
    if (lane == 0) {
      S.VF[j] = VFj;
      // mixed path: a polyhedron inside one cell's fluid or empty part has
      // an exact V_F; any other carries FP32 error (launch_repair)
      if constexpr (sizeof(G) == 4) S.fexact[j] = (wh != 0 && !err) ? 1 : 0;
    }
  }
  if (lane == 0) {
    if (n_trunc) atomicAdd(S.cnt + kNTrunc, n_trunc);
    if (n_over) atomicAdd(S.cnt + kNOverflow, n_over);
    if (n_deg) atomicAdd(S.cnt + kNDegen, n_deg);
    if (n_edge) atomicAdd(S.cnt + kNEdgeOn, n_edge);
  }
}

// export of candidate lists (parity of the overlap lists): the same union as
// the flux kernel streams, unfiltered, written ascending
constexpr int kCandCap = 256;
__global__ void k_candidates(DevMesh M, const int32_t* faces, int n, int64_t cap, int32_t* out,
                             int32_t* counts) {
  __shared__ int32_t lists[kWarps][kCandCap];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* list = lists[wib];
  for (int w = blockIdx.x * kWarps + wib; w < n; w += gridDim.x * kWarps) {
    const int j = faces[w];
    const int own = M.own[j], nbr = M.nbr[j];
    const int64_t a0 = M.nb_ptr[own];
    const int na = (int)(M.nb_ptr[own + 1] - a0);
    int m = 0;
    for (int pass = 0; pass < 2; ++pass) {
      const int c0 = pass == 0 ? own : nbr;
      if (c0 < 0) break;
      const int64_t b0 = M.nb_ptr[c0];
      const int nb = (int)(M.nb_ptr[c0 + 1] - b0) + 1;
      for (int base = 0; base < nb; base += 32) {
        const int idx = base + lane;
        int k = -1;
        if (idx < nb) k = (idx == nb - 1) ? c0 : M.nb[b0 + idx];
        bool keep = k >= 0;
        if (keep && pass == 1) keep = !(k == own || sorted_contains(M.nb + a0, na, k));
        const unsigned bal = __ballot_sync(GVOF_FULL, keep);
        if (keep) {
          const int pos = m + __popc(bal & ((1u << lane) - 1u));
          if (pos < kCandCap) list[pos] = k;
        }
        m += __popc(bal);
      }
    }
    if (lane == 0) counts[w] = m;
    const int mm = m < kCandCap ? m : kCandCap;
    __syncwarp();
    int e[kCandCap / 32], r[kCandCap / 32];
    for (int q = 0; q < kCandCap / 32; ++q) {
      const int idx = lane + 32 * q;
      e[q] = idx < mm ? list[idx] : 0;
      r[q] = 0;
    }
    for (int t = 0; t < mm; ++t) {
      const int v = list[t];
      for (int q = 0; q < kCandCap / 32; ++q) r[q] += (v < e[q]);
    }
    __syncwarp();
    for (int q = 0; q < kCandCap / 32; ++q)
      if (lane + 32 * q < mm && r[q] < cap) out[w * cap + r[q]] = e[q];
    __syncwarp();
  }
}

template <typename G, int KIND>
__global__ void k_polyhedra(DevMesh M, GeoView<G> Gv, const GridParam* gp, const double* srate,
                            const int32_t* faces, int n, double* verts, int32_t* counts) {
  __shared__ Poly<G> polys[kWarps];
  __shared__ FaceFrame<G> wfr[kWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Poly<G>& P = polys[wib];
  FaceFrame<G>& fr = wfr[wib];
  for (int w = blockIdx.x * kWarps + wib; w < n; w += gridDim.x * kWarps) {
    const int j = faces[w];
    const GridParam& gq = gp[grid_of(M.face_off, M.n_grids, j)];
    const double Vd = srate[j] * gq.g * gq.dt;
    const bool ok = build_polyhedron<G, KIND>(M, Gv, gq, j, Vd, P, fr, lane);
    if (lane == 0) counts[w] = ok ? fr.I : -1;
    if (ok && lane < base_verts<KIND>(fr.I)) {
      const double L = (double)fr.L;
      const int64_t o = ((int64_t)w * VOF_MAX_POLY_VERTS + lane) * 3;
      verts[o + 0] = absd(fr.cx) + L * (double)P.bx[lane];
      verts[o + 1] = absd(fr.cy) + L * (double)P.by[lane];
      verts[o + 2] = absd(fr.cz) + L * (double)P.bz[lane];
    }
    __syncwarp();
  }
}

}  // namespace

namespace {
template <typename G, int KIND>
void prebuild_launch(const vof_ctx* c, cudaStream_t s) {
  k_prebuild<G, KIND><<<kSMs * 8, 128, 0, s>>>(mesh_view(c), geo_view<G>(c), state_view(c));
}
template <typename G>
void prebuild_launch_kind(const vof_ctx* c, cudaStream_t s) {
  switch (c->opt.flux_polyhedron) {
    case VOF_FLUX_EMFPA: prebuild_launch<G, VOF_FLUX_EMFPA>(c, s); break;
    case VOF_FLUX_NMFPA: prebuild_launch<G, VOF_FLUX_NMFPA>(c, s); break;
    default: prebuild_launch<G, VOF_FLUX_FMFPA>(c, s); break;
  }
}
template <typename G, int KIND, int GW>
void flux_launch(const vof_ctx* c, int grid, cudaStream_t s) {
  if constexpr (GW == 16) {
    // eight half-warp polyhedra per block: ask for the largest shared-memory
    // carve-out so that as many blocks stay resident as with whole warps
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(k_flux<G, KIND, GW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      set = true;
    }
  }
  k_flux<G, KIND, GW><<<grid, kWarps * 32, 0, s>>>(mesh_view(c), geo_view<G>(c), state_view(c));
}
template <typename G>
void flux_launch_kind(const vof_ctx* c, int grid, cudaStream_t s) {
  // two faces per warp where the context allows it (FMFPA and NMFPA on
  // grids of convex cells with at most 16 faces and faces of at most 5
  // nodes; see vof_options.faces_per_warp)
  const bool half = c->faces_per_warp == 2;
  switch (c->opt.flux_polyhedron) {
    case VOF_FLUX_EMFPA: flux_launch<G, VOF_FLUX_EMFPA, 32>(c, grid, s); break;
    case VOF_FLUX_NMFPA:
      if (half) flux_launch<G, VOF_FLUX_NMFPA, 16>(c, grid, s);
      else flux_launch<G, VOF_FLUX_NMFPA, 32>(c, grid, s);
      break;
    default:
      if (half) flux_launch<G, VOF_FLUX_FMFPA, 16>(c, grid, s);
      else flux_launch<G, VOF_FLUX_FMFPA, 32>(c, grid, s);
      break;
  }
}
template <typename G, int KIND>
void polyhedra_launch(const vof_ctx* c, const int32_t* faces, int n, double* verts, int32_t* counts,
                      cudaStream_t s) {
  k_polyhedra<G, KIND><<<kSMs, kWarps * 32, 0, s>>>(mesh_view(c), geo_view<G>(c), c->gp_d, c->srate,
                                                    faces, n, verts, counts);
}
template <typename G>
void polyhedra_launch_kind(const vof_ctx* c, const int32_t* faces, int n, double* verts,
                           int32_t* counts, cudaStream_t s) {
  switch (c->opt.flux_polyhedron) {
    case VOF_FLUX_EMFPA: polyhedra_launch<G, VOF_FLUX_EMFPA>(c, faces, n, verts, counts, s); break;
    case VOF_FLUX_NMFPA: polyhedra_launch<G, VOF_FLUX_NMFPA>(c, faces, n, verts, counts, s); break;
    default: polyhedra_launch<G, VOF_FLUX_FMFPA>(c, faces, n, verts, counts, s); break;
  }
}
}  // namespace

bool prebuild_lists(const vof_ctx* c) { return c->fm_cand != nullptr && c->fm_use > 0; }

cudaError_t launch_prebuild(const vof_ctx* c, cudaStream_t s) {
  if (c->opt.precision != VOF_PREC_MIXED) {
    prebuild_launch_kind<double>(c, s);
    return cudaGetLastError();
  }
  prebuild_launch_kind<float>(c, s);
  if (prebuild_lists(c)) {
    const DevMesh m = mesh_view(c);
    const GeoView<float> g = geo_view<float>(c);
    const DevState st = state_view(c);
    const int grid = kSMs * 8;  // 16 face groups per block
    switch (c->opt.flux_polyhedron) {
      case VOF_FLUX_EMFPA: k_candlist<float, VOF_FLUX_EMFPA><<<grid, kListWarps * 32, 0, s>>>(m, g, st); break;
      case VOF_FLUX_NMFPA: k_candlist<float, VOF_FLUX_NMFPA><<<grid, kListWarps * 32, 0, s>>>(m, g, st); break;
      default: k_candlist<float, VOF_FLUX_FMFPA><<<grid, kListWarps * 32, 0, s>>>(m, g, st); break;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_flux(const vof_ctx* c, cudaStream_t s) {
  const int grid = c->flux_blocks > 0 ? c->flux_blocks : kSMs * GVOF_FLUX_MINB;
  const cudaError_t e = cudaMemsetAsync(c->cnt + kFluxNext, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (c->opt.precision == VOF_PREC_MIXED) flux_launch_kind<float>(c, grid, s);
  else flux_launch_kind<double>(c, grid, s);
  return cudaGetLastError();
}

cudaError_t launch_candidates(const vof_ctx* c, const int32_t* faces, int n, int64_t cap,
                              int32_t* out, int32_t* counts, cudaStream_t s) {
  k_candidates<<<kSMs, kWarps * 32, 0, s>>>(mesh_view(c), faces, n, cap, out, counts);
  return cudaGetLastError();
}

cudaError_t launch_polyhedra(const vof_ctx* c, const int32_t* faces, int n, double* verts,
                             int32_t* counts, cudaStream_t s) {
  if (c->opt.precision == VOF_PREC_MIXED) polyhedra_launch_kind<float>(c, faces, n, verts, counts, s);
  else polyhedra_launch_kind<double>(c, faces, n, verts, counts, s);
  return cudaGetLastError();
}

}  // namespace gvof

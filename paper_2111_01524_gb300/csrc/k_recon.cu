// PLIC reconstruction of the interfacial cells: LSGIR normal (Sec. 2.1.1,
// Eqs. eq:lsgir1, eq:lsgir2, lsgir-beta) and the volume-enforcing plane
// constant (Sec. 2.1, Eq. plic-eq), optionally refined by the LSFIR outer
// iteration (Sec. 2.1.2). One warp per interfacial cell.
//
// Plane constant, GPU design: V(C) = vol(cell ∩ {n.x + C >= 0}) is evaluated
// by clipping each face of the cell (Sutherland-Hodgman) and summing the
// divergence-theorem fan with the origin placed ON the cutting plane, so the
// cap polygon contributes nothing and is never built. Lane v evaluates V at
// the breakpoint C_v = -n.x_v of vertex v; warp max/min reductions give the
// bracket between consecutive breakpoints, where V is exactly a cubic in C.
// Two more evaluations inside the bracket fix the cubic, whose root is found
// by safeguarded Newton iteration. Each round of evaluations spreads its
// (sample, face) pairs over the lanes.
// Precision: the FP64 path works in double. The mixed path works in FP32 in
// cell-local coordinates scaled by V^(-1/3) (absolute positions as (hi, lo)
// float pairs); for cells with F or 1 - F below 1e-3, where an FP32 cut
// volume is too coarse to place the plane, it takes the corner closed form
// (FP32 relative to the corner) or the FP64 bracket. Axis-aligned boxes of
// the mixed LSGIR path take the cuboid closed form of box_plane.cuh instead,
// one thread per cell after the normals (k_box_constant).
#include "vof_common.cuh"
#include "box_plane.cuh"

namespace gvof {
namespace {

// blocks per SM the register allocation must allow (64 registers a thread
// at 8: twice the resident warps of an unbounded allocation, measured faster)
#ifndef GVOF_RECON_MINB
#define GVOF_RECON_MINB 8
#endif

constexpr int kWarps = 4;
constexpr int kMaxCellFaces = 32;
constexpr int kMaxCellEntries = 128;
constexpr double kNear01 = 1e-3;

template <typename P>
struct LoopSmem {
  P x[kMaxCellEntries], y[kMaxCellEntries], z[kMaxCellEntries];  // outward face loops
};

struct ReconSmem {
  union {
    LoopSmem<double> d;
    LoopSmem<float> f;
  };
  int vid[kMaxCellEntries];  // vertex id of each loop entry
  int fs[kMaxCellFaces + 1];
  int corner[4];             // neighbours of the extreme vertex
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GVOF_FULL, v, o);
  return v;
}

__device__ __forceinline__ const LoopSmem<double>& loops(const ReconSmem& S, double) { return S.d; }
__device__ __forceinline__ const LoopSmem<float>& loops(const ReconSmem& S, float) { return S.f; }
__device__ __forceinline__ LoopSmem<double>& loops_w(ReconSmem& S, double) { return S.d; }
__device__ __forceinline__ LoopSmem<float>& loops_w(ReconSmem& S, float) { return S.f; }

// adds to vol six times the contribution of face f to the volume of the
// part of the cell where n.x + C >= 0 (scaled cell-local frame): the face
// loop clipped to the half-space and fanned from a point of the plane, so
// that the cap the cut would close contributes nothing
template <typename P>
__device__ void face_cut(const ReconSmem& S, int f, P nx, P ny, P nz, P C, P& vol) {
  const LoopSmem<P>& Lp = loops(S, P(0));
  const P ox = -C * nx, oy = -C * ny, oz = -C * nz;  // a point of the plane
  const int b = S.fs[f], L = S.fs[f + 1] - b;
  P ax = Lp.x[b + L - 1] - ox, ay = Lp.y[b + L - 1] - oy, az = Lp.z[b + L - 1] - oz;
  P pa = nx * ax + ny * ay + nz * az;
  int ne = 0;
  P q0x = 0, q0y = 0, q0z = 0, qpx = 0, qpy = 0, qpz = 0;
  for (int k = 0; k < L; ++k) {
    const P bx = Lp.x[b + k] - ox, by = Lp.y[b + k] - oy, bz = Lp.z[b + k] - oz;
    const P pb = nx * bx + ny * by + nz * bz;
    const bool ia = pa >= P(0), ib = pb >= P(0);
    // emit the clipped polygon's points in order; fan from the first
    for (int e = 0; e < 2; ++e) {
      P px, py, pz;
      if (e == 0) {
        if (ia == ib) continue;
        // interpolate from the inside end, as the face on the other side of
        // this edge does, so both compute the same point bit for bit
        if (ia) {
          const P t = pa / (pa - pb);
          px = ax + t * (bx - ax); py = ay + t * (by - ay); pz = az + t * (bz - az);
        } else {
          const P t = pb / (pb - pa);
          px = bx + t * (ax - bx); py = by + t * (ay - by); pz = bz + t * (az - bz);
        }
      } else {
        if (!ib) continue;
        px = bx; py = by; pz = bz;
      }
      if (ne == 0) { q0x = px; q0y = py; q0z = pz; }
      else if (ne >= 2)
        vol += q0x * (qpy * pz - qpz * py) + q0y * (qpz * px - qpx * pz) + q0z * (qpx * py - qpy * px);
      qpx = px; qpy = py; qpz = pz;
      ++ne;
    }
    ax = bx; ay = by; az = bz; pa = pb;
  }
}

// V(C_s) for ns samples at once: lane (s, g), s = lane % ns, clips the faces
// g, g + G, ... (G = 32 / ns groups) at the lane's C (that of its sample s),
// and the groups' partial sums are added in a fixed order; every lane returns
// the volume of its sample. FP64 keeps one lane per sample (G = 1), so that
// its sums are formed in the order of the plain face-by-face evaluation.
template <typename P>
__device__ P cut_volumes(const ReconSmem& S, int nfc, P nx, P ny, P nz, P C, int ns, int lane) {
  const int G = sizeof(P) == 8 ? 1 : 32 / ns;
  const int s = lane % ns, g = lane / ns;
  P part = P(0);
  if (g < G)
    for (int f = g; f < nfc; f += G) face_cut<P>(S, f, nx, ny, nz, C, part);
  P tot = P(0);
  for (int gg = 0; gg < G; ++gg) tot += __shfl_sync(GVOF_FULL, part, s + ns * gg);
  return tot / P(6);
}

// plane constant (cell-local, scaled) for target volume T; lane v < ncv
// holds the projection s_v = n.x_v of vertex v
template <typename P>
__device__ P plane_constant(const ReconSmem& S, int nfc, int ncv, P s_lane, P nx, P ny, P nz, P T,
                            int lane) {
  const bool has = lane < ncv;
  const P Cv = has ? -s_lane : P(0);
  // V at the breakpoint of every vertex, lanes (vertex, face group)
  const P Vall = cut_volumes<P>(S, nfc, nx, ny, nz, __shfl_sync(GVOF_FULL, Cv, lane % ncv), ncv, lane);
  const P Vv = has ? Vall : P(0);
  // bracket [Ca, Cb]: largest breakpoint with V <= T, smallest with V >= T
  P Ca = (has && Vv <= T) ? Cv : P(-1e30), Va = Vv;
  P Cb = (has && Vv >= T) ? Cv : P(1e30), Vb = Vv;
  for (int o = 16; o > 0; o >>= 1) {
    const P c2 = __shfl_xor_sync(GVOF_FULL, Ca, o), v2 = __shfl_xor_sync(GVOF_FULL, Va, o);
    if (c2 > Ca) { Ca = c2; Va = v2; }
    const P c3 = __shfl_xor_sync(GVOF_FULL, Cb, o), v3 = __shfl_xor_sync(GVOF_FULL, Vb, o);
    if (c3 < Cb) { Cb = c3; Vb = v3; }
  }
  if (Va == T || !(Cb > Ca)) return Ca;
  if (Vb == T) return Cb;
  // V is a cubic on [Ca, Cb]: sample at 1/3 (even lanes) and 2/3 (odd lanes)
  const P Cm = Ca + (Cb - Ca) * ((lane & 1) == 0 ? P(1) / P(3) : P(2) / P(3));
  const P Vm = cut_volumes<P>(S, nfc, nx, ny, nz, Cm, 2, lane);
  const P y0 = Va, y3 = Vb;
  const P y1 = __shfl_sync(GVOF_FULL, Vm, 0), y2 = __shfl_sync(GVOF_FULL, Vm, 1);
  // Newton forward form in s = 3 (C - Ca) / (Cb - Ca), s in [0, 3]
  const P d1 = y1 - y0, d2 = y2 - P(2) * y1 + y0, d3 = y3 - P(3) * y2 + P(3) * y1 - y0;
  P lo = P(0), hi = P(3);
  P s = P(3) * (T - y0) / (y3 - y0);
  const P tol = P(3) * (sizeof(P) == 8 ? P(2e-16) : P(2e-7));
  for (int it = 0; it < 50; ++it) {
    const P p = y0 + s * (d1 + (s - P(1)) * (P(0.5) * d2 + (s - P(2)) * d3 / P(6)));
    const P dp = d1 + d2 * (s - P(0.5)) + d3 * (P(3) * s * s - P(6) * s + P(2)) / P(6);
    if (p < T) lo = s; else hi = s;
    P sn = (dp > P(0)) ? s - (p - T) / dp : P(0.5) * (lo + hi);
    if (!(sn > lo && sn < hi)) sn = P(0.5) * (lo + hi);
    const bool done = fabs(sn - s) <= tol || hi - lo <= tol;
    s = sn;
    if (done) break;
  }
  return Ca + (s / P(3)) * (Cb - Ca);
}

// Closed-form plane constant when the fluid (or, for F > 1/2, the empty)
// region is the corner of an extreme vertex with three edges: between that
// vertex and the next breakpoint the region is the tetrahedron cut off the
// three edges e_i, of volume D^3 |det(e1,e2,e3)| / (6 |n.e1 n.e2 n.e3|) at
// plane distance D from the vertex, so D = cbrt(6 T |n.e1 n.e2 n.e3| / |det|).
// FP64; returns false when the corner does not apply (the bracketing method
// is used then). Needs the loops' vertex ids in smem and s_lane = n.(x_v-xc).
// the vertices that follow v in the cell's outward loops (its edge
// neighbours), up to 4 into Sm.corner; returns how many there are
__device__ int vertex_neighbours(const DevMesh& M, ReconSmem& Sm, int c, int v, int lane) {
  const int nent = Sm.fs[M.cf_ptr[c + 1] - M.cf_ptr[c]];
  int found = 0;
  for (int base = 0; base < nent; base += 32) {
    const int e = base + lane;
    int nb = -1;
    if (e < nent && Sm.vid[e] == v) {
      int f = 0;
      while (Sm.fs[f + 1] <= e) ++f;
      const int nxt = (e + 1 == Sm.fs[f + 1]) ? Sm.fs[f] : e + 1;
      nb = Sm.vid[nxt];
    }
    const unsigned bal = __ballot_sync(GVOF_FULL, nb >= 0);
    if (nb >= 0) {
      const int pos = found + __popc(bal & ((1u << lane) - 1u));
      if (pos < 4) Sm.corner[pos] = nb;
    }
    found += __popc(bal);
  }
  __syncwarp();
  return found;
}

// Prism form of the corner solution, for an extreme projection shared by
// exactly two vertices v1, v1b joined by an edge e3 that lies in the plane
// (a cell extruded along e3, e.g. a quasi-2D grid's): when both ends have
// their other two edges e1, e2 equal, the region within distance D of the
// top is the corner triangle (v1, v1 + D/a1 e1, v1 + D/a2 e2) swept along
// e3, of volume D^2 |det(e1, e2, e3)| / (2 a1 a2), a_i = n.e_i towards the
// region, valid up to the next breakpoint k3. E holds the edges' coordinate
// differences (v1's edges to its neighbours; the same for v1b), in the
// units of a (absolute for FP64, scaled for FP32). Returns D or -1.
template <typename T>
__device__ T prism_distance(const T e1[3], const T e2[3], const T e3[3], T a1, T a2, T vol, T dmax,
                            T tiny) {
  const T det = fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                     e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]));
  if (!(a1 > tiny && a2 > tiny) || !(det > T(0))) return T(-1);
  if (!(vol <= dmax * dmax * det / (T(2) * a1 * a2))) return T(-1);
  return sqrt(T(2) * vol * a1 * a2 / det);
}

// the prism form (prism_distance) of corner_constant, out of line: it runs
// for cells whose extreme projection is shared by two vertices
__device__ __noinline__ bool corner_prism(const DevMesh& M, ReconSmem& Sm, int c, int ncv, int vl,
                                          double key, double k1, int v1, double sgn, bool low,
                                          double nx, double ny, double nz, double F, double Vc,
                                          int lane, double* Cout) {
  const unsigned tie = __ballot_sync(GVOF_FULL, lane < ncv && key == k1);
  if (__popc(tie) != 2) return false;
  const int la = __ffs(tie) - 1, lb = 31 - __clz(tie);
  const int va = __shfl_sync(GVOF_FULL, vl, la), vb = __shfl_sync(GVOF_FULL, vl, lb);
  const int v1b = va == v1 ? vb : va;
  double k3 = (lane < ncv && key < k1) ? key : -1e300;
  for (int o = 16; o > 0; o >>= 1) k3 = fmax(k3, __shfl_xor_sync(GVOF_FULL, k3, o));
  if (vertex_neighbours(M, Sm, c, v1, lane) != 3) return false;
  int na[3] = {Sm.corner[0], Sm.corner[1], Sm.corner[2]};
  __syncwarp();
  if (vertex_neighbours(M, Sm, c, v1b, lane) != 3) return false;
  const int nbv[3] = {Sm.corner[0], Sm.corner[1], Sm.corner[2]};
  __syncwarp();
  // v1's edges: e3 to v1b, e1 and e2 to the others
  int j = 0;
  double E[2][3], e3[3] = {M.x[v1b] - M.x[v1], M.y[v1b] - M.y[v1], M.z[v1b] - M.z[v1]};
  for (int i = 0; i < 3; ++i) {
    if (na[i] == v1b) continue;
    if (j == 2) return false;
    E[j][0] = M.x[na[i]] - M.x[v1]; E[j][1] = M.y[na[i]] - M.y[v1]; E[j][2] = M.z[na[i]] - M.z[v1];
    ++j;
  }
  if (j != 2) return false;
  // v1b's other two edges must be the same vectors
  int matched = 0;
  for (int i = 0; i < 3; ++i) {
    if (nbv[i] == v1) continue;
    const double d0 = M.x[nbv[i]] - M.x[v1b], d1 = M.y[nbv[i]] - M.y[v1b], d2 = M.z[nbv[i]] - M.z[v1b];
    for (int q = 0; q < 2; ++q)
      if (d0 == E[q][0] && d1 == E[q][1] && d2 == E[q][2]) matched |= 1 << q;
  }
  if (matched != 3) return false;
  const double a1 = -sgn * (nx * E[0][0] + ny * E[0][1] + nz * E[0][2]);
  const double a2 = -sgn * (nx * E[1][0] + ny * E[1][1] + nz * E[1][2]);
  const double hs = cbrt(Vc), hsc = 1.0 / hs;
  const double T = (low ? F : 1.0 - F) * Vc;
  const double D = prism_distance<double>(E[0], E[1], e3, a1, a2, T, (k1 - k3) / hsc, 1e-9 * hs);
  if (!(D >= 0.0)) return false;
  const double s_top = k1 / hsc;
  *Cout = low ? (D - s_top) : (s_top - D);
  return true;
}

__device__ bool corner_constant(const DevMesh& M, ReconSmem& Sm, int c, int ncv, int vl,
                                double s_lane, double nx, double ny, double nz, double F,
                                double Vc, int lane, double* Cout) {
  const bool low = F <= 0.5;  // fluid corner at the top vertex, else empty corner at the bottom
  const double key = lane < ncv ? (low ? s_lane : -s_lane) : -1e300;
  // extreme vertex (largest key) and the next breakpoint
  double k1 = key, k2 = -1e300;
  int v1 = vl;
  for (int o = 16; o > 0; o >>= 1) {
    const double ok1 = __shfl_xor_sync(GVOF_FULL, k1, o), ok2 = __shfl_xor_sync(GVOF_FULL, k2, o);
    const int ov1 = __shfl_xor_sync(GVOF_FULL, v1, o);
    if (ok1 > k1 || (ok1 == k1 && ov1 < v1)) {
      k2 = fmax(k1, ok2);
      k1 = ok1;
      v1 = ov1;
    } else {
      k2 = fmax(k2, ok1);
    }
  }
  const double sgn = low ? 1.0 : -1.0;
  if (k2 == k1) return corner_prism(M, Sm, c, ncv, vl, key, k1, v1, sgn, low, nx, ny, nz, F, Vc, lane, Cout);
  // neighbours of v1: the entry after v1 in every outward loop
  const int found = vertex_neighbours(M, Sm, c, v1, lane);
  if (found != 3) return false;
  double e[3][3], a[3];
  for (int i = 0; i < 3; ++i) {
    const int w = Sm.corner[i];
    e[i][0] = M.x[w] - M.x[v1]; e[i][1] = M.y[w] - M.y[v1]; e[i][2] = M.z[w] - M.z[v1];
    a[i] = -sgn * (nx * e[i][0] + ny * e[i][1] + nz * e[i][2]);  // > 0 along the edges
  }
  const double det = fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                          e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                          e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]));
  const double hs = cbrt(Vc);
  if (!(a[0] > 1e-9 * hs && a[1] > 1e-9 * hs && a[2] > 1e-9 * hs) || !(det > 0.0)) return false;
  const double prod = a[0] * a[1] * a[2];
  const double T = (low ? F : 1.0 - F) * Vc;
  const double hsc = 1.0 / cbrt(Vc);
  // breakpoint distance in absolute units (s was formed in scaled units)
  const double D2 = (k1 - k2) / hsc;
  if (!(T <= D2 * D2 * D2 * det / (6.0 * prod))) return false;
  const double D = cbrt(6.0 * T * prod / det);
  const double s_top = k1 / hsc;  // key of the extreme vertex, absolute units
  // low: fluid = {s >= s_top - D}, C = D - s_top; high: empty = {s <= s_bot + D}
  *Cout = low ? (D - s_top) : (s_top - D);
  return true;
}

// FP32 form of corner_constant for the mixed path: the same closed form in
// the scaled cell-local frame, edges from the (hi, lo) positions. The mixed
// path stores its plane constants in FP32, whose rounding (a few 1e-8 of the
// cell size) bounds what an FP64 root would add. Returns the scaled C.
// the prism form (prism_distance) of corner_constant32, out of line
template <typename G>
__device__ __noinline__ bool corner_prism32(const DevMesh& M, const GeoView<G>& Gv, ReconSmem& Sm, int c,
                                            int ncv, int vl, float key, float k1, int v1, float sgn,
                                            bool low, float nx, float ny, float nz, double F, float Vs,
                                            float sc, int lane, float* Cout) {
  const unsigned tie = __ballot_sync(GVOF_FULL, lane < ncv && key == k1);
  if (__popc(tie) != 2) return false;
  const int la = __ffs(tie) - 1, lb = 31 - __clz(tie);
  const int va = __shfl_sync(GVOF_FULL, vl, la), vb = __shfl_sync(GVOF_FULL, vl, lb);
  const int v1b = va == v1 ? vb : va;
  float k3 = (lane < ncv && key < k1) ? key : -1e30f;
  for (int o = 16; o > 0; o >>= 1) k3 = fmaxf(k3, __shfl_xor_sync(GVOF_FULL, k3, o));
  if (vertex_neighbours(M, Sm, c, v1, lane) != 3) return false;
  int na[3] = {Sm.corner[0], Sm.corner[1], Sm.corner[2]};
  __syncwarp();
  if (vertex_neighbours(M, Sm, c, v1b, lane) != 3) return false;
  const int nbv[3] = {Sm.corner[0], Sm.corner[1], Sm.corner[2]};
  __syncwarp();
  int j = 0;
  float E[2][3];
  const float e3[3] = {(float)(rel(Gv.vx[v1b], Gv.vx[v1]) * sc), (float)(rel(Gv.vy[v1b], Gv.vy[v1]) * sc),
                       (float)(rel(Gv.vz[v1b], Gv.vz[v1]) * sc)};
  for (int i = 0; i < 3; ++i) {
    if (na[i] == v1b) continue;
    if (j == 2) return false;
    E[j][0] = (float)(rel(Gv.vx[na[i]], Gv.vx[v1]) * sc);
    E[j][1] = (float)(rel(Gv.vy[na[i]], Gv.vy[v1]) * sc);
    E[j][2] = (float)(rel(Gv.vz[na[i]], Gv.vz[v1]) * sc);
    ++j;
  }
  if (j != 2) return false;
  int matched = 0;
  for (int i = 0; i < 3; ++i) {
    if (nbv[i] == v1) continue;
    const float d0 = (float)(rel(Gv.vx[nbv[i]], Gv.vx[v1b]) * sc),
                d1 = (float)(rel(Gv.vy[nbv[i]], Gv.vy[v1b]) * sc),
                d2 = (float)(rel(Gv.vz[nbv[i]], Gv.vz[v1b]) * sc);
    for (int q = 0; q < 2; ++q)
      if (d0 == E[q][0] && d1 == E[q][1] && d2 == E[q][2]) matched |= 1 << q;
  }
  if (matched != 3) return false;
  const float a1 = -sgn * (nx * E[0][0] + ny * E[0][1] + nz * E[0][2]);
  const float a2 = -sgn * (nx * E[1][0] + ny * E[1][1] + nz * E[1][2]);
  const float T = (float)((low ? F : 1.0 - F) * (double)Vs);
  const float D = prism_distance<float>(E[0], E[1], e3, a1, a2, T, k1 - k3, 1e-6f);
  if (!(D >= 0.f)) return false;
  *Cout = low ? (D - k1) : (k1 - D);
  return true;
}

template <typename G>
__device__ bool corner_constant32(const DevMesh& M, const GeoView<G>& Gv, ReconSmem& Sm, int c, int ncv,
                                  int vl, float s_lane, float nx, float ny, float nz, double F, float Vs,
                                  float sc, int lane, float* Cout) {
  const bool low = F <= 0.5;  // fluid corner at the top vertex, else empty corner at the bottom
  const float key = lane < ncv ? (low ? s_lane : -s_lane) : -1e30f;
  float k1 = key, k2 = -1e30f;
  int v1 = vl;
  for (int o = 16; o > 0; o >>= 1) {
    const float ok1 = __shfl_xor_sync(GVOF_FULL, k1, o), ok2 = __shfl_xor_sync(GVOF_FULL, k2, o);
    const int ov1 = __shfl_xor_sync(GVOF_FULL, v1, o);
    if (ok1 > k1 || (ok1 == k1 && ov1 < v1)) {
      k2 = fmaxf(k1, ok2);
      k1 = ok1;
      v1 = ov1;
    } else {
      k2 = fmaxf(k2, ok1);
    }
  }
  const float sgn = low ? 1.f : -1.f;
  if (k2 == k1) return corner_prism32<G>(M, Gv, Sm, c, ncv, vl, key, k1, v1, sgn, low, nx, ny, nz, F, Vs, sc, lane, Cout);
  const int found = vertex_neighbours(M, Sm, c, v1, lane);
  if (found != 3) return false;
  float e[3][3], a[3];
  for (int i = 0; i < 3; ++i) {
    const int w = Sm.corner[i];
    e[i][0] = rel(Gv.vx[w], Gv.vx[v1]) * sc;
    e[i][1] = rel(Gv.vy[w], Gv.vy[v1]) * sc;
    e[i][2] = rel(Gv.vz[w], Gv.vz[v1]) * sc;
    a[i] = -sgn * (nx * e[i][0] + ny * e[i][1] + nz * e[i][2]);  // > 0 along the edges
  }
  const float det = fabsf(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                          e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                          e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]));
  if (!(a[0] > 1e-6f && a[1] > 1e-6f && a[2] > 1e-6f) || !(det > 0.f)) return false;
  const float prod = a[0] * a[1] * a[2];
  const float T = (float)((low ? F : 1.0 - F) * (double)Vs);
  const float D2 = k1 - k2;
  if (!(T <= D2 * D2 * D2 * det / (6.f * prod))) return false;
  const float D = cbrtf(6.f * T * prod / det);
  *Cout = low ? (D - k1) : (k1 - D);
  return true;
}

// load the cell's outward face loops (cell-local, scaled) in precision P
template <typename P, typename G>
__device__ void load_loops(const DevMesh& M, const GeoView<G>& Gv, ReconSmem& Sm, int c,
                           typename Prec<G>::A xc, typename Prec<G>::A yc,
                           typename Prec<G>::A zc, double sc, int nfc, int lane) {
  LoopSmem<P>& Lp = loops_w(Sm, P(0));
  const int64_t f0 = M.cf_ptr[c];
  int fid = 0, len = 0;
  bool out = true;
  if (lane < nfc) {
    const int fs = M.cf[f0 + lane];
    out = fs >= 0;
    fid = out ? fs : ~fs;
    len = (int)(M.fptr[fid + 1] - M.fptr[fid]);
  }
  int off = len;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(GVOF_FULL, off, d);
    if (lane >= d) off += t;
  }
  if (lane < nfc) {
    Sm.fs[lane + 1] = off;
    off -= len;
    if (lane == 0) Sm.fs[0] = 0;
    const int64_t b = M.fptr[fid];
    for (int i = 0; i < len; ++i) {
      const int v = M.fvert[b + (out ? i : len - 1 - i)];
      Sm.vid[off + i] = v;
      if (sizeof(P) == sizeof(G)) {
        Lp.x[off + i] = (P)(rel(Gv.vx[v], xc) * (G)sc);
        Lp.y[off + i] = (P)(rel(Gv.vy[v], yc) * (G)sc);
        Lp.z[off + i] = (P)(rel(Gv.vz[v], zc) * (G)sc);
      } else {  // FP64 loops from (hi, lo) pairs: exact differences in double
        Lp.x[off + i] = (P)(((double)M.x[v] - (double)M.ccx[c]) * sc);
        Lp.y[off + i] = (P)(((double)M.y[v] - (double)M.ccy[c]) * sc);
        Lp.z[off + i] = (P)(((double)M.z[v] - (double)M.ccz[c]) * sc);
      }
    }
  }
  __syncwarp();
}

// Vertex average of the PLIC polygon n.x + C = 0 (Sec. 2.1.2) in the
// scaled cell-local frame of the loops last loaded in precision P: each loop
// edge whose ends lie strictly on opposite sides gives its crossing, formed
// from the end with the lower vertex id so that the two loops through an
// edge give the same point; a cell vertex exactly on the plane (lane v < ncv
// holds vertex v at (vx, vy, vz), formed as the loops form their vertices)
// counts as often as an edge, twice. Returns (0, 0, 0), the centroid, when
// the plane misses the cell.
template <typename P>
__device__ void plic_centre(const ReconSmem& S, int nfc, P nx, P ny, P nz, P C, bool vact, P vx,
                            P vy, P vz, int lane, P& cx, P& cy, P& cz) {
  const LoopSmem<P>& L = loops(S, P(0));
  P sx = P(0), sy = P(0), sz = P(0);
  int cnt = 0;
  if (lane < nfc) {
    const int b = S.fs[lane], e = S.fs[lane + 1];
    for (int i = b; i < e; ++i) {
      const int j = (i + 1 < e) ? i + 1 : b;
      const bool sw = S.vid[j] < S.vid[i];
      const int a = sw ? j : i, o = sw ? i : j;
      const P pa = nx * L.x[a] + ny * L.y[a] + nz * L.z[a] + C;
      const P po = nx * L.x[o] + ny * L.y[o] + nz * L.z[o] + C;
      if ((pa > P(0) && po < P(0)) || (pa < P(0) && po > P(0))) {
        const P t = pa / (pa - po);
        sx += L.x[a] + t * (L.x[o] - L.x[a]);
        sy += L.y[a] + t * (L.y[o] - L.y[a]);
        sz += L.z[a] + t * (L.z[o] - L.z[a]);
        ++cnt;
      }
    }
  }
  if (vact && nx * vx + ny * vy + nz * vz + C == P(0)) {
    sx += P(2) * vx; sy += P(2) * vy; sz += P(2) * vz;
    cnt += 2;
  }
  sx = warp_sum(sx); sy = warp_sum(sy); sz = warp_sum(sz);
  cnt = warp_sum(cnt);
  if (cnt == 0) {
    cx = cy = cz = P(0);
  } else {
    cx = sx / (P)cnt; cy = sy / (P)cnt; cz = sz / (P)cnt;
  }
}

// PLIC centre of cell c from the loops in precision P (scaled frame, C the
// scaled constant, h the cell size that unscales it), stored for LSFIR: FP64
// path absolute, mixed path as FP32 offsets from the centroid
template <typename P, typename G, bool kMixed>
__device__ void store_centre(const DevMesh& M, const DevState& S, const ReconSmem& Sm, int c, int nfc,
                             P nx, P ny, P nz, P C, bool vact, P vx, P vy, P vz, double h, int lane) {
  P cx, cy, cz;
  plic_centre<P>(Sm, nfc, nx, ny, nz, C, vact, vx, vy, vz, lane, cx, cy, cz);
  if (lane == 0) {
    if constexpr (kMixed) {
      S.lxr[c] = (float)((double)cx * h); S.lyr[c] = (float)((double)cy * h); S.lzr[c] = (float)((double)cz * h);
    } else {
      S.lxp[c] = M.ccx[c] + (double)cx * h;
      S.lyp[c] = M.ccy[c] + (double)cy * h;
      S.lzp[c] = M.ccz[c] + (double)cz * h;
    }
  }
}

// eigen-decomposition of the symmetric 3x3 matrix A by cyclic Jacobi
// rotations (each zeroes A[p][q]): on return the diagonal holds the
// eigenvalues and the columns of V the eigenvectors
template <typename T>
__device__ void sym3_jacobi(T A[3][3], T V[3][3]) {
  const T tol = sizeof(T) == 8 ? T(1e-32) : T(1e-14);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = T(i == j);
  for (int sweep = 0; sweep < 64; ++sweep) {
    const T off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const T dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= tol * dia || off == T(0)) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
      if (A[p][q] == T(0)) continue;
      const T th = (A[q][q] - A[p][p]) / (T(2) * A[p][q]);
      const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
      const T cs = T(1) / sqrt(t * t + T(1)), sn = t * cs;
      // A <- J^T A J, V <- V J with J = I except J_pp = J_qq = cs, J_pq = sn, J_qp = -sn
      T Ap[3], Aq[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Ap[k] = A[k][p] * cs - A[k][q] * sn;  // column p of A J
        Aq[k] = A[k][p] * sn + A[k][q] * cs;  // column q of A J
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) { A[k][p] = Ap[k]; A[k][q] = Aq[k]; }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Ap[k] = cs * A[p][k] - sn * A[q][k];  // row p of J^T (A J)
        Aq[k] = sn * A[p][k] + cs * A[q][k];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) { A[p][k] = Ap[k]; A[q][k] = Aq[k]; }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T vp = V[k][p] * cs - V[k][q] * sn, vq = V[k][p] * sn + V[k][q] * cs;
        V[k][p] = vp; V[k][q] = vq;
      }
    }
  }
}

// Minimum-norm least-squares gradient of a singular LSGIR system (Sec.
// 2.1.1), e.g. on a quasi-2D grid one cell thick, where every neighbour
// offset lies in the plane: the pseudo-inverse of A^T A over its eigenvalues
// above a relative threshold (FP64 1e-12, FP32 1e-6) applied to A^T b;
// (1, 0, 0) if that leaves nothing. Out of line: it is the rare branch.
template <typename G>
__device__ __noinline__ void lsgir_pinv(G m00, G m01, G m02, G m11, G m12, G m22, G r0, G r1, G r2,
                                        G& gx, G& gy, G& gz) {
  G A[3][3] = {{m00, m01, m02}, {m01, m11, m12}, {m02, m12, m22}}, V[3][3];
  sym3_jacobi(A, V);
  const G top = fmax(A[0][0], fmax(A[1][1], A[2][2]));
  const G thr = (sizeof(G) == 8 ? G(1e-12) : G(1e-6)) * top;
  gx = gy = gz = G(0);
  for (int k = 0; k < 3; ++k) {
    if (!(A[k][k] > thr)) continue;
    const G c = (V[0][k] * r0 + V[1][k] * r1 + V[2][k] * r2) / A[k][k];
    gx += c * V[0][k]; gy += c * V[1][k]; gz += c * V[2][k];
  }
  if (!(gx * gx + gy * gy + gz * gz > G(0))) { gx = 1; gy = 0; gz = 0; }
}

// LSFIR normal update of outer iteration io (Sec. 2.1.2): the plane through
// the cell's PLIC centre x that minimises sum_k w_k (n.(x_k - x))^2 over the
// valid neighbours (interfacial node neighbours whose normal is within 45
// degrees of the cell's, both of the previous iteration), w_k =
// |x_k - x|^-2.5: the eigenvector of the smallest eigenvalue of
// sum_k w_k d_k d_k^T (distances scaled by the cell size, which leaves it
// unchanged), oriented like the previous normal. The cell takes it if it
// turns its normal by less than lim = 30 degrees / io (kept otherwise, and
// with fewer than two valid neighbours or collinear centres); the result
// goes to the band-position buffer, so that every cell is decided from the
// previous iteration, and the largest accepted turn to S.lturn[io]. Nothing
// is done once an earlier iteration turned no normal by tol or more.
// Work split: a warp gathers and reduces the sums of 32 cells one after the
// other (lanes over neighbours), then lane i solves cell i's eigenproblem,
// so the FP64 solve runs once per cell (the FP64 pipe processes a warp
// instruction at the same cost whatever its active lanes). The sums and the
// solve are FP64 in both paths: in FP32 the eigenvector of a nearly
// degenerate matrix drifts from the FP64 result; the mixed path forms the
// distances and weights in FP32 (from (hi, lo) centroids and FP32 centre
// offsets), the FP64 path in FP64.
template <typename G, bool kMixed>
__global__ void __launch_bounds__(kWarps * 32) k_lsfir_normals(DevMesh M, GeoView<G> Gv, DevState S,
                                                            int io, double lim, double tol) {
  if (io > 1 && __longlong_as_double((long long)S.lturn[io - 1]) < tol) return;
  __shared__ double sums[kWarps][6][32];
  __shared__ int nval[kWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned n_ic = (unsigned)S.cnt[kNIcells];
  const double cos45 = sqrt(0.5);
  for (unsigned base = (blockIdx.x * kWarps + wib) * 32u; base < n_ic;
       base += gridDim.x * kWarps * 32u) {
    const int nb = (int)min(32u, n_ic - base);
    for (int i = 0; i < nb; ++i) {
      const int c = S.icells[base + i];
      const double ncx = Gv.pnx[c], ncy = Gv.pny[c], ncz = Gv.pnz[c];
      const G sc = G(1) / cbrt(Gv.cvol[c]);
      double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
      int nv = 0;
      const int64_t q0 = M.nb_ptr[c], q1 = M.nb_ptr[c + 1];
      for (int64_t q = q0 + lane; q < q1; q += 32) {
        const int k = M.nb[q];
        if (S.tc[k] != 0) continue;
        if (!(ncx * (double)Gv.pnx[k] + ncy * (double)Gv.pny[k] + ncz * (double)Gv.pnz[k] > cos45))
          continue;
        G dx, dy, dz;
        if constexpr (kMixed) {
          dx = (rel(Gv.ccx[k], Gv.ccx[c]) + (S.lxr[k] - S.lxr[c])) * sc;
          dy = (rel(Gv.ccy[k], Gv.ccy[c]) + (S.lyr[k] - S.lyr[c])) * sc;
          dz = (rel(Gv.ccz[k], Gv.ccz[c]) + (S.lzr[k] - S.lzr[c])) * sc;
        } else {
          dx = (S.lxp[k] - S.lxp[c]) * sc;
          dy = (S.lyp[k] - S.lyp[c]) * sc;
          dz = (S.lzp[k] - S.lzp[c]) * sc;
        }
        const double ex = dx, ey = dy, ez = dz;
        double wk;  // |d|^-2.5: FP32 on the mixed path (its distances are FP32)
        if constexpr (kMixed) {
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 > 0.f)) continue;
          wk = 1.f / (r2 * sqrtf(sqrtf(r2)));
        } else {
          const double r2 = ex * ex + ey * ey + ez * ez;
          if (!(r2 > 0.0)) continue;
          wk = 1.0 / (r2 * sqrt(sqrt(r2)));
        }
        m00 += wk * ex * ex; m01 += wk * ex * ey; m02 += wk * ex * ez;
        m11 += wk * ey * ey; m12 += wk * ey * ez; m22 += wk * ez * ez;
        ++nv;
      }
      m00 = warp_sum(m00); m01 = warp_sum(m01); m02 = warp_sum(m02);
      m11 = warp_sum(m11); m12 = warp_sum(m12); m22 = warp_sum(m22);
      nv = warp_sum(nv);
      if (lane == i) {
        sums[wib][0][i] = m00; sums[wib][1][i] = m01; sums[wib][2][i] = m02;
        sums[wib][3][i] = m11; sums[wib][4][i] = m12; sums[wib][5][i] = m22;
        nval[wib][i] = nv;
      }
    }
    __syncwarp();
    double turned = 0.0;
    if (lane < nb) {
      const unsigned w = base + lane;
      const int c = S.icells[w];
      const double ncx = Gv.pnx[c], ncy = Gv.pny[c], ncz = Gv.pnz[c];
      double vx = ncx, vy = ncy, vz = ncz;
      if (nval[wib][lane] >= 2) {
        const double m00 = sums[wib][0][lane], m01 = sums[wib][1][lane], m02 = sums[wib][2][lane];
        const double m11 = sums[wib][3][lane], m12 = sums[wib][4][lane], m22 = sums[wib][5][lane];
        double A[3][3] = {{m00, m01, m02}, {m01, m11, m12}, {m02, m12, m22}}, V[3][3];
        sym3_jacobi(A, V);
        int lo = 0;
        if (A[1][1] < A[lo][lo]) lo = 1;
        if (A[2][2] < A[lo][lo]) lo = 2;
        const int i1 = lo == 0 ? 1 : 0, i2 = lo == 2 ? 1 : 2;
        const double e1 = A[i1][i1], e2 = A[i2][i2];
        const double mid = e1 < e2 ? e1 : e2, top = e1 < e2 ? e2 : e1;
        if (mid - A[lo][lo] > 1e-12 * top) {
          double ex = V[0][lo], ey = V[1][lo], ez = V[2][lo];
          const double en = sqrt(ex * ex + ey * ey + ez * ez);
          const double sg = (ex * ncx + ey * ncy + ez * ncz < 0.0) ? -1.0 : 1.0;
          ex = sg * ex / en; ey = sg * ey / en; ez = sg * ez / en;
          const double cx = ncy * ez - ncz * ey, cy = ncz * ex - ncx * ez, cz = ncx * ey - ncy * ex;
          const double ang = atan2(sqrt(cx * cx + cy * cy + cz * cz), ncx * ex + ncy * ey + ncz * ez);
          if (ang < lim) {
            vx = ex; vy = ey; vz = ez;
            turned = ang;
          }
        }
      }
      if constexpr (kMixed) {
        S.lnx32[w] = (float)vx; S.lny32[w] = (float)vy; S.lnz32[w] = (float)vz;
      } else {
        S.lnx[w] = vx; S.lny[w] = vy; S.lnz[w] = vz;
      }
    }
    // the batch's largest accepted turn, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) turned = fmax(turned, __shfl_xor_sync(GVOF_FULL, turned, o));
    if (lane == 0 && turned > 0.0)
      atomicMax(S.lturn + io, (unsigned long long)__double_as_longlong(turned));
    __syncwarp();
  }
}

// MODE 0: LSGIR normal and plane constant. MODE 1: the same, then the
// PLIC centre for LSFIR, and the per-iteration turn slots cleared. MODE 2
// (LSFIR outer iteration io): the normal accepted by k_lsfir_normals, its
// plane constant and PLIC centre; nothing once an earlier iteration turned
// no normal by tol or more.
// the next interfacial cell for this warp, dealt from a counter like the flux
// kernel's faces (cells near F = 0 or 1 take the corner form, the others the
// bracketed solve: their costs differ)
__device__ __forceinline__ unsigned next_cell(const DevState& S, int lane) {
  unsigned w = 0u;
  if (lane == 0) w = (unsigned)atomicAdd(S.cnt + kReconNext, 1ull);
  return __shfl_sync(GVOF_FULL, w, 0);
}

template <typename G, bool kMixed, int MODE>
__global__ void __launch_bounds__(kWarps * 32, GVOF_RECON_MINB) k_reconstruct(DevMesh M, GeoView<G> Gv, DevState S,
                                                             double beta, int io, double tol) {
  if constexpr (MODE == 2) {
    if (io > 1 && __longlong_as_double((long long)S.lturn[io - 1]) < tol) return;
  }
  if constexpr (MODE == 1) {
    if (blockIdx.x == 0 && threadIdx.x <= kMaxLsfirIter) S.lturn[threadIdx.x] = 0ull;
  }
  __shared__ ReconSmem smem[kWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  ReconSmem& Sm = smem[wib];
  const unsigned n_ic = (unsigned)S.cnt[kNIcells];
  const bool beta15 = (beta == 1.5);
  const G gbeta = (G)beta;
  for (unsigned w = next_cell(S, lane); w < n_ic; w = next_cell(S, lane)) {
    const int c = S.icells[w];
    const typename Prec<G>::A xc = Gv.ccx[c], yc = Gv.ccy[c], zc = Gv.ccz[c];
    const G V = Gv.cvol[c];
    const G hc = cbrt(V), sc = G(1) / hc;
    const double Fc = S.F[c];
    const G Fcg = (G)Fc;
    G nx, ny, nz;
    if constexpr (MODE == 2) {
      if constexpr (kMixed) {
        nx = S.lnx32[w]; ny = S.lny32[w]; nz = S.lnz32[w];
      } else {
        nx = S.lnx[w]; ny = S.lny[w]; nz = S.lnz[w];
      }
    } else {
    // ---- LSGIR: weighted least squares for grad F (Sec. 2.1.1)
    G m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0, r0 = 0, r1 = 0, r2 = 0;
    const int64_t q0 = M.nb_ptr[c], q1 = M.nb_ptr[c + 1];
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const int k = M.nb[q];
      const G dx = rel(Gv.ccx[k], xc) * sc, dy = rel(Gv.ccy[k], yc) * sc, dz = rel(Gv.ccz[k], zc) * sc;
      const G d2 = dx * dx + dy * dy + dz * dz;
      const G w2 = beta15 ? G(1) / (d2 * sqrt(d2)) : pow(d2, -gbeta);  // w_k^2 = |d|^(-2 beta)
      const G df = (G)S.F[k] - Fcg;
      m00 += w2 * dx * dx; m01 += w2 * dx * dy; m02 += w2 * dx * dz;
      m11 += w2 * dy * dy; m12 += w2 * dy * dz; m22 += w2 * dz * dz;
      r0 += w2 * dx * df; r1 += w2 * dy * df; r2 += w2 * dz * df;
    }
    m00 = warp_sum(m00); m01 = warp_sum(m01); m02 = warp_sum(m02);
    m11 = warp_sum(m11); m12 = warp_sum(m12); m22 = warp_sum(m22);
    r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2);
    // (A^T A) g = A^T b by the adjugate (symmetric 3x3); only the direction
    // of g matters
    const G a00 = m11 * m22 - m12 * m12, a01 = m02 * m12 - m01 * m22, a02 = m01 * m12 - m02 * m11;
    const G a11 = m00 * m22 - m02 * m02, a12 = m01 * m02 - m00 * m12, a22 = m00 * m11 - m01 * m01;
    const G det = m00 * a00 + m01 * a01 + m02 * a02;
    const G tr = m00 + m11 + m22;
    G gx, gy, gz;
    if (fabs(det) > G(1e-12) * tr * tr * tr) {
      gx = a00 * r0 + a01 * r1 + a02 * r2;
      gy = a01 * r0 + a11 * r1 + a12 * r2;
      gz = a02 * r0 + a12 * r1 + a22 * r2;
      if (det < G(0)) { gx = -gx; gy = -gy; gz = -gz; }
    } else {
      lsgir_pinv<G>(m00, m01, m02, m11, m12, m22, r0, r1, r2, gx, gy, gz);
    }
    G gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (!(gn > G(0))) { gx = 1; gy = 0; gz = 0; gn = 1; }
    nx = gx / gn; ny = gy / gn; nz = gz / gn;
    }

    if constexpr (MODE == 0 && kMixed) {
      if (M.convex[c] == 2) {
        // an axis-aligned box: its plane constant is taken by
        // k_box_constant, one thread per cell
        if (lane == 0) {
          S.nx[c] = (double)nx; S.ny[c] = (double)ny; S.nz[c] = (double)nz;
          if (kMixed) { S.nx32[c] = (float)nx; S.ny32[c] = (float)ny; S.nz32[c] = (float)nz; }
        }
        __syncwarp();
        continue;
      }
    }
    // ---- plane constant
    const int nfc = (int)(M.cf_ptr[c + 1] - M.cf_ptr[c]);
    const int64_t v0 = M.cv_ptr[c];
    const int ncv = (int)(M.cv_ptr[c + 1] - v0);
    const int vl = lane < ncv ? M.cv[v0 + lane] : M.cv[v0];
    double Cout;
    const bool near01 = Fc < kNear01 || Fc > 1.0 - kNear01;
    if (kMixed && near01) {
      // FP32 corner closed form
      load_loops<G, G>(M, Gv, Sm, c, xc, yc, zc, (double)sc, nfc, lane);
      const G s = nx * rel(Gv.vx[vl], xc) * sc + ny * rel(Gv.vy[vl], yc) * sc +
                  nz * rel(Gv.vz[vl], zc) * sc;
      float C32c;
      if (corner_constant32(M, Gv, Sm, c, ncv, vl, (float)s, (float)nx, (float)ny, (float)nz, Fc,
                            (float)(V * sc * sc * sc), (float)sc, lane, &C32c)) {
        Cout = (double)(C32c * (float)hc);
        if (lane == 0) {
          S.nx[c] = (double)nx; S.ny[c] = (double)ny; S.nz[c] = (double)nz; S.C[c] = Cout;
          S.nx32[c] = (float)nx; S.ny32[c] = (float)ny; S.nz32[c] = (float)nz; S.C32[c] = (float)Cout;
        }
        if constexpr (MODE >= 1) {
          const G vx = rel(Gv.vx[vl], xc) * sc, vy = rel(Gv.vy[vl], yc) * sc, vz = rel(Gv.vz[vl], zc) * sc;
          store_centre<G, G, kMixed>(M, S, Sm, c, nfc, nx, ny, nz, (G)C32c, lane < ncv, vx, vy, vz,
                                     (double)hc, lane);
        }
        __syncwarp();
        continue;
      }
    }
    if (!kMixed) {
      // FP64 closed form when the fluid / empty region is a vertex corner
      const double hcd = cbrt(M.cvol[c]), scd = 1.0 / hcd;
      load_loops<double, G>(M, Gv, Sm, c, xc, yc, zc, scd, nfc, lane);
      const double nxd = nx, nyd = ny, nzd = nz;
      const double s = nxd * (M.x[vl] - M.ccx[c]) * scd + nyd * (M.y[vl] - M.ccy[c]) * scd +
                       nzd * (M.z[vl] - M.ccz[c]) * scd;
      if (corner_constant(M, Sm, c, ncv, vl, s, nxd, nyd, nzd, Fc, M.cvol[c], lane, &Cout)) {
        if (lane == 0) {
          S.nx[c] = nxd; S.ny[c] = nyd; S.nz[c] = nzd; S.C[c] = Cout;
          if (kMixed) {
            S.nx32[c] = (float)nx; S.ny32[c] = (float)ny; S.nz32[c] = (float)nz; S.C32[c] = (float)Cout;
          }
        }
        if constexpr (MODE >= 1) {
          const double vx = (M.x[vl] - M.ccx[c]) * scd, vy = (M.y[vl] - M.ccy[c]) * scd,
                       vz = (M.z[vl] - M.ccz[c]) * scd;
          store_centre<double, G, kMixed>(M, S, Sm, c, nfc, nxd, nyd, nzd, Cout * scd, lane < ncv, vx,
                                          vy, vz, hcd, lane);
        }
        __syncwarp();
        continue;
      }
    }
    if (kMixed && near01) {
      const double hcd = cbrt(M.cvol[c]), scd = 1.0 / hcd;
      load_loops<double, G>(M, Gv, Sm, c, xc, yc, zc, scd, nfc, lane);
      const double nxd = nx, nyd = ny, nzd = nz;
      const double s = nxd * (M.x[vl] - M.ccx[c]) * scd + nyd * (M.y[vl] - M.ccy[c]) * scd +
                       nzd * (M.z[vl] - M.ccz[c]) * scd;
      const double T = Fc * M.cvol[c] * scd * scd * scd;
      const double Cs = plane_constant<double>(Sm, nfc, ncv, s, nxd, nyd, nzd, T, lane);
      Cout = Cs * hcd;
      if constexpr (MODE >= 1) {
        const double vx = (M.x[vl] - M.ccx[c]) * scd, vy = (M.y[vl] - M.ccy[c]) * scd,
                     vz = (M.z[vl] - M.ccz[c]) * scd;
        store_centre<double, G, kMixed>(M, S, Sm, c, nfc, nxd, nyd, nzd, Cs, lane < ncv, vx, vy, vz,
                                        hcd, lane);
      }
    } else {
      load_loops<G, G>(M, Gv, Sm, c, xc, yc, zc, (double)sc, nfc, lane);
      const G s = nx * rel(Gv.vx[vl], xc) * sc + ny * rel(Gv.vy[vl], yc) * sc +
                  nz * rel(Gv.vz[vl], zc) * sc;
      const G T = Fcg * V * sc * sc * sc;
      const G Cs = plane_constant<G>(Sm, nfc, ncv, s, nx, ny, nz, T, lane);
      Cout = (double)(Cs * hc);
      if constexpr (MODE >= 1) {
        const G vx = rel(Gv.vx[vl], xc) * sc, vy = rel(Gv.vy[vl], yc) * sc, vz = rel(Gv.vz[vl], zc) * sc;
        store_centre<G, G, kMixed>(M, S, Sm, c, nfc, nx, ny, nz, Cs, lane < ncv, vx, vy, vz, (double)hc,
                                   lane);
      }
    }
    if (lane == 0) {
      S.nx[c] = (double)nx; S.ny[c] = (double)ny; S.nz[c] = (double)nz; S.C[c] = Cout;
      if (kMixed) {
        S.nx32[c] = (float)nx; S.ny32[c] = (float)ny; S.nz32[c] = (float)nz; S.C32[c] = (float)Cout;
      }
    }
    __syncwarp();
  }
}

// plane constants of the interfacial box cells of the mixed path, one
// thread per cell; the root g in FP32 (relative to the corner it bounds, so
// a nearly full or empty cell keeps its precision), C from it in FP64; the
// normals come from k_reconstruct
__global__ void k_box_constant(DevMesh M, DevState S) {
  const int64_t n = (int64_t)S.cnt[kNIcells];
  const int64_t nc = M.nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = S.icells[i];
    if (M.convex[c] != 2) continue;
    const double F = S.F[c];
    const double n0 = S.nx[c], n1 = S.ny[c], n2 = S.nz[c];
    const double lx = M.bb[c], ly = M.bb[nc + c], lz = M.bb[2 * nc + c];
    const double hx = M.bb[3 * nc + c], hy = M.bb[4 * nc + c], hz = M.bb[5 * nc + c];
    const double a0 = fabs(n0 * (hx - lx)), a1 = fabs(n1 * (hy - ly)), a2 = fabs(n2 * (hz - lz));
    const double Sa = a0 + a1 + a2;
    const double d = n0 * (0.5 * (lx + hx) - M.ccx[c]) + n1 * (0.5 * (ly + hy) - M.ccy[c]) +
                     n2 * (0.5 * (lz + hz) - M.ccz[c]);
    const BoxSlopes B = box_slopes((float)(a0 / Sa), (float)(a1 / Sa), (float)(a2 / Sa));
    const float v = (float)(F < 0.5 ? F : 1.0 - F);
    const double g = (double)box_root(v, B);
    const double C = (F >= 0.5 ? Sa * (0.5 - g) : Sa * (g - 0.5)) - d;
    S.C[c] = C;
    S.C32[c] = (float)C;
  }
}

}  // namespace

int reconstruct_launch_count(const vof_ctx* c) {
  // LSGIR: the warp kernel, and in the mixed path the box cells' constants
  if (c->opt.reconstruction == VOF_RECON_LSFIR) return 1 + 2 * c->opt.lsfir_max_iter;
  return c->opt.precision == VOF_PREC_MIXED ? 2 : 1;
}

namespace {
template <typename G, bool kMixed>
cudaError_t reconstruct_launches(const vof_ctx* c, cudaStream_t s) {
  const int grid = c->recon_blocks > 0 ? c->recon_blocks : kSMs * 8;
  const DevMesh m = mesh_view(c);
  const GeoView<G> g = geo_view<G>(c);
  const DevState st = state_view(c);
  const double beta = c->opt.beta;
  // each k_reconstruct launch deals its cells from a fresh counter
  auto reset = [&]() {
    return cudaMemsetAsync(c->cnt + kReconNext, 0, sizeof(unsigned long long), s);
  };
  cudaError_t e = reset();
  if (e != cudaSuccess) return e;
  if (c->opt.reconstruction != VOF_RECON_LSFIR) {
    k_reconstruct<G, kMixed, 0><<<grid, kWarps * 32, 0, s>>>(m, g, st, beta, 0, 0.0);
    if (kMixed) k_box_constant<<<kSMs * 4, 128, 0, s>>>(m, st);
    return cudaGetLastError();
  }
  // LSFIR (Sec. 2.1.2): LSGIR start, then the outer iterations; each
  // launch skips its work once the iteration has converged, so the launch
  // sequence is fixed (and can be captured in a graph)
  const double lim30 = 30.0 * 3.14159265358979323846 / 180.0, tol = c->opt.lsfir_tol;
  k_reconstruct<G, kMixed, 1><<<grid, kWarps * 32, 0, s>>>(m, g, st, beta, 0, tol);
  for (int io = 1; io <= c->opt.lsfir_max_iter; ++io) {
    k_lsfir_normals<G, kMixed><<<kSMs * 8, kWarps * 32, 0, s>>>(m, g, st, io, lim30 / io, tol);
    if ((e = reset()) != cudaSuccess) return e;
    k_reconstruct<G, kMixed, 2><<<grid, kWarps * 32, 0, s>>>(m, g, st, beta, io, tol);
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_reconstruct(const vof_ctx* c, cudaStream_t s) {
  if (c->opt.precision == VOF_PREC_MIXED) return reconstruct_launches<float, true>(c, s);
  return reconstruct_launches<double, false>(c, s);
}

}  // namespace gvof

// Face fluxes of the active faces (Sec. 2.2): FMFPA flux polyhedron
// (Sec. 2.2.2) of each tag-0 face, truncated by the half-spaces of every
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
// (ping-pong), and the base polyhedron that is restored per candidate cell.
// FP64 path: G = double. Mixed path: G = float in face-local coordinates
// scaled by 1/sqrt(A_face); the volumes are summed in FP64.
#include "vof_common.cuh"

namespace gvof {
namespace {

constexpr int kWarps = 4;
constexpr int MAXI = kMaxFaceVerts;   // face vertices
constexpr int NB = 2 * MAXI + 1;      // base polyhedron vertices / faces
constexpr int NV = 80;                // vertex table capacity
constexpr int NF = 32;                // face capacity (one lane each)
constexpr int LM = 32;                // loop length capacity
constexpr int NR = 32;                // new vertices per clip
constexpr int NCAND = 64;             // surviving candidate cells per face

template <typename G>
struct __align__(16) Poly {
  G vx[NV], vy[NV], vz[NV];
  G phi[NV];
  G bx[NB], by[NB], bz[NB];  // base polyhedron
  int32_t cand[NCAND];
  uint8_t fv[2][NF][LM];
  uint8_t flen[2][NF];
  uint8_t ra[NR], rb[NR];    // cut-edge records: inside vertex, outside vertex
  int8_t capnext[NR];
  uint8_t newid[NV];
};

template <typename T>
__device__ __forceinline__ T wsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GVOF_FULL, v, o);
  return v;
}
__device__ __forceinline__ double wmin(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(GVOF_FULL, v, o));
  return v;
}
__device__ __forceinline__ double wmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(GVOF_FULL, v, o));
  return v;
}

struct PolyState {
  int nv, nf, cur;
};

// restore the FMFPA polyhedron: x_0..x_{I-1}, back-traced I..2I-1, apex 2I;
// faces: the cell face, I side quads, I bottom triangles (Sec. 2.2.2)
template <typename G>
__device__ void restore_base(Poly<G>& P, PolyState& st, int I, int lane) {
  const int nvb = 2 * I + 1;
  if (lane < nvb) {
    P.vx[lane] = P.bx[lane]; P.vy[lane] = P.by[lane]; P.vz[lane] = P.bz[lane];
  }
  if (lane < nvb) {
    uint8_t* o = P.fv[0][lane];
    if (lane == 0) {
      for (int i = 0; i < I; ++i) o[i] = (uint8_t)i;
      P.flen[0][0] = (uint8_t)I;
    } else if (lane <= I) {
      int i = lane - 1, ip = (i + 1 == I) ? 0 : i + 1;
      o[0] = (uint8_t)ip; o[1] = (uint8_t)i; o[2] = (uint8_t)(I + i); o[3] = (uint8_t)(I + ip);
      P.flen[0][lane] = 4;
    } else {
      int i = lane - 1 - I, ip = (i + 1 == I) ? 0 : i + 1;
      o[0] = (uint8_t)(I + ip); o[1] = (uint8_t)(I + i); o[2] = (uint8_t)(2 * I);
      P.flen[0][lane] = 3;
    }
  }
  st.nv = nvb;
  st.nf = nvb;
  st.cur = 0;
  __syncwarp();
}

// drop unreferenced vertices and renumber (keeps room for a clip)
template <typename G>
__device__ void compact(Poly<G>& P, PolyState& st, int lane) {
  for (int v = lane; v < NV; v += 32) P.newid[v] = 0;
  __syncwarp();
  if (lane < st.nf) {
    const uint8_t* lp = P.fv[st.cur][lane];
    for (int k = 0; k < P.flen[st.cur][lane]; ++k) P.newid[lp[k]] = 1;
  }
  __syncwarp();
  // exclusive prefix over the marks (NV <= 96: three per lane)
  int m[3], s = 0;
  for (int r = 0; r < 3; ++r) {
    int v = lane * 3 + r;
    m[r] = (v < st.nv) ? P.newid[v] : 0;
    s += m[r];
  }
  int incl = s;
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(GVOF_FULL, incl, d);
    if (lane >= d) incl += t;
  }
  int total = __shfl_sync(GVOF_FULL, incl, 31);
  int base = incl - s;
  G x[3], y[3], z[3];
  for (int r = 0; r < 3; ++r) {
    int v = lane * 3 + r;
    if (v < st.nv && m[r]) { x[r] = P.vx[v]; y[r] = P.vy[v]; z[r] = P.vz[v]; }
  }
  __syncwarp();
  for (int r = 0; r < 3; ++r) {
    int v = lane * 3 + r;
    if (v < st.nv && m[r]) {
      P.vx[base] = x[r]; P.vy[base] = y[r]; P.vz[base] = z[r];
      P.newid[v] = (uint8_t)base;
      ++base;
    }
  }
  __syncwarp();
  if (lane < st.nf) {
    uint8_t* lp = P.fv[st.cur][lane];
    for (int k = 0; k < P.flen[st.cur][lane]; ++k) lp[k] = P.newid[lp[k]];
  }
  st.nv = total;
  __syncwarp();
}

// clip the closed surface by the half-space a.x + b >= 0.
// returns 0: unchanged, 1: clipped, 2: empty. err bit0: capacity overflow.
template <typename G>
__device__ int clip(Poly<G>& P, PolyState& st, G a0, G a1, G a2, G b, int lane, unsigned& err) {
  if (st.nv > NV - NR) compact(P, st, lane);
  for (int v = lane; v < st.nv; v += 32) P.phi[v] = a0 * P.vx[v] + a1 * P.vy[v] + a2 * P.vz[v] + b;
  __syncwarp();
  const int cur = st.cur, nf = st.nf, nv = st.nv;
  bool has_in = false, has_out = false;
  int nexit = 0, L = 0;
  const uint8_t* lp = P.fv[cur][lane < NF ? lane : 0];
  if (lane < nf) {
    L = P.flen[cur][lane];
    bool prev = P.phi[lp[L - 1]] >= G(0);
    for (int k = 0; k < L; ++k) {
      bool in = P.phi[lp[k]] >= G(0);
      has_in |= in;
      has_out |= !in;
      nexit += (prev && !in);
      prev = in;
    }
  }
  const unsigned bin = __ballot_sync(GVOF_FULL, has_in);
  const unsigned bout = __ballot_sync(GVOF_FULL, has_out);
  if (bout == 0) return 0;
  if (bin == 0) { st.nf = 0; return 2; }
  int incl = nexit;
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(GVOF_FULL, incl, d);
    if (lane >= d) incl += t;
  }
  const int total = __shfl_sync(GVOF_FULL, incl, 31);
  const int off = incl - nexit;
  if (total > NR || nv + total > NV) { err |= 1u; st.nf = 0; return 2; }
  // new vertices on the cut edges, created by the face leaving the half-space
  if (lane < nf && nexit) {
    int r = off;
    for (int k = 0; k < L; ++k) {
      const int va = lp[k], vb = lp[(k + 1 == L) ? 0 : k + 1];
      const G pa = P.phi[va], pb = P.phi[vb];
      if (pa >= G(0) && !(pb >= G(0))) {
        const G t = pa / (pa - pb);
        const int id = nv + r;
        P.vx[id] = P.vx[va] + t * (P.vx[vb] - P.vx[va]);
        P.vy[id] = P.vy[va] + t * (P.vy[vb] - P.vy[va]);
        P.vz[id] = P.vz[va] + t * (P.vz[vb] - P.vz[va]);
        P.ra[r] = (uint8_t)va;
        P.rb[r] = (uint8_t)vb;
        P.capnext[r] = -1;
        ++r;
      }
    }
  }
  __syncwarp();
  const int nxt = cur ^ 1;
  const int slot = __popc(bin & ((1u << lane) - 1u));
  bool bad = false;
  if (lane < nf && has_in) {
    uint8_t* op = P.fv[nxt][slot];
    int k0 = 0;
    while (!(P.phi[lp[k0]] >= G(0))) ++k0;
    int n = 0, pend = -1;
    for (int s = 0; s < L; ++s) {
      int k = k0 + s;
      if (k >= L) k -= L;
      const int k1 = (k + 1 == L) ? 0 : k + 1;
      const int va = lp[k], vb = lp[k1];
      const bool ia = P.phi[va] >= G(0), ib = P.phi[vb] >= G(0);
      if (ia) { if (n < LM) op[n] = (uint8_t)va; ++n; }
      if (ia && !ib) {
        int r = -1;
        for (int q = off; q < off + nexit; ++q)
          if (P.ra[q] == va && P.rb[q] == vb) { r = q; break; }
        if (r < 0) { bad = true; break; }
        if (n < LM) op[n] = (uint8_t)(nv + r);
        ++n;
        pend = r;
      } else if (!ia && ib) {
        int r = -1;
        for (int q = 0; q < total; ++q)
          if (P.ra[q] == vb && P.rb[q] == va) { r = q; break; }
        if (r < 0 || pend < 0) { bad = true; break; }
        if (n < LM) op[n] = (uint8_t)(nv + r);
        ++n;
        P.capnext[r] = (int8_t)pend;  // cap edge: entry -> preceding exit
      }
    }
    if (n > LM) bad = true;
    P.flen[nxt][slot] = (uint8_t)(n > LM ? LM : n);
  }
  if (__any_sync(GVOF_FULL, bad)) { err |= 1u; st.nf = 0; return 2; }
  __syncwarp();
  // cap loops
  int nfo = __popc(bin);
  if (lane == 0) {
    unsigned vis = 0u;
    for (int r = 0; r < total; ++r) {
      if ((vis >> r) & 1u) continue;
      if (nfo >= NF) { err |= 1u; break; }
      uint8_t* op = P.fv[nxt][nfo];
      int n = 0, s = r;
      while (s >= 0 && !((vis >> s) & 1u) && n < LM) {
        vis |= 1u << s;
        op[n++] = (uint8_t)(nv + s);
        s = P.capnext[s];
      }
      if (s != r) err |= 1u;  // open chain: inconsistent topology
      if (n >= 3) { P.flen[nxt][nfo] = (uint8_t)n; ++nfo; }
    }
  }
  nfo = __shfl_sync(GVOF_FULL, nfo, 0);
  st.nv = nv + total;
  st.nf = nfo;
  st.cur = nxt;
  __syncwarp();
  return 1;
}

// signed volume of the surface: each lane fans one face loop
template <typename G>
__device__ double volume(const Poly<G>& P, const PolyState& st, int lane) {
  G acc = G(0);
  if (st.nf > 0) {
    const int o = P.fv[st.cur][0][0];
    const G ox = P.vx[o], oy = P.vy[o], oz = P.vz[o];
    if (lane < st.nf) {
      const uint8_t* lp = P.fv[st.cur][lane];
      const int L = P.flen[st.cur][lane];
      const G x0 = P.vx[lp[0]] - ox, y0 = P.vy[lp[0]] - oy, z0 = P.vz[lp[0]] - oz;
      G px = P.vx[lp[1]] - ox, py = P.vy[lp[1]] - oy, pz = P.vz[lp[1]] - oz;
      for (int k = 2; k < L; ++k) {
        const G qx = P.vx[lp[k]] - ox, qy = P.vy[lp[k]] - oy, qz = P.vz[lp[k]] - oz;
        acc += x0 * (py * qz - pz * qy) + y0 * (pz * qx - px * qz) + z0 * (px * qy - py * qx);
        px = qx; py = qy; pz = qz;
      }
    }
  }
  return wsum((double)acc) / 6.0;
}

struct FluxParams {
  Vel vel;
  double g;   // time factor at t + dt/2
  double dt;
};

struct FaceFrame {
  double cx, cy, cz, L, sc;
  int I;
  double lo[3], hi[3];  // absolute bounding box of the polyhedron
  int degenerate, edgeon;
};

// FMFPA construction (Sec. 2.2.2) into P.b*: side plane i contains edge i
// and is parallel to the velocity at the edge centre; back-traced vertex i
// is the projection of the streak-line point x_i - dt u_i (Eq.
// streak-line2) on the line where side planes i-1 and i meet; the centroid
// of the back-traced loop moves along the face normal by the closed-form
// amount that makes the signed volume equal V_d.
template <typename G>
__device__ bool build_fmfpa(const DevMesh& M, const FluxParams& p, int j, double Vd, Poly<G>& P,
                            FaceFrame& fr, int lane) {
  const int64_t fb = M.fptr[j];
  const int I = (int)(M.fptr[j + 1] - fb);
  fr.I = I;
  if (I > MAXI || I < 3) return false;
  fr.cx = M.fcx[j]; fr.cy = M.fcy[j]; fr.cz = M.fcz[j];
  const double A = M.fa[j];
  fr.L = sqrt(A);
  fr.sc = 1.0 / fr.L;
  const double nxd = M.fnx[j], nyd = M.fny[j], nzd = M.fnz[j];
  const bool act = lane < I;
  const int vi = act ? M.fvert[fb + lane] : M.fvert[fb];
  const double X = M.x[vi], Y = M.y[vi], Z = M.z[vi];
  const int nxt = (lane + 1 >= I) ? 0 : lane + 1;
  const int prv = (lane == 0) ? I - 1 : lane - 1;
  const double Xn = __shfl_sync(GVOF_FULL, X, nxt), Yn = __shfl_sync(GVOF_FULL, Y, nxt),
               Zn = __shfl_sync(GVOF_FULL, Z, nxt);
  // velocities at the vertex and at the centre of edge (i, i+1), times dt,
  // in face-local scaled units
  G ux, uy, uz, ex_u, ey_u, ez_u;
  vel0<G>(p.vel, (G)X, (G)Y, (G)Z, ux, uy, uz);
  vel0<G>(p.vel, (G)(0.5 * (X + Xn)), (G)(0.5 * (Y + Yn)), (G)(0.5 * (Z + Zn)), ex_u, ey_u, ez_u);
  const G k = (G)(p.g * p.dt * fr.sc);
  ux *= k; uy *= k; uz *= k; ex_u *= k; ey_u *= k; ez_u *= k;
  const G lx = (G)((X - fr.cx) * fr.sc), ly = (G)((Y - fr.cy) * fr.sc), lz = (G)((Z - fr.cz) * fr.sc);
  const G lxn = __shfl_sync(GVOF_FULL, lx, nxt), lyn = __shfl_sync(GVOF_FULL, ly, nxt),
          lzn = __shfl_sync(GVOF_FULL, lz, nxt);
  const G ex = lxn - lx, ey = lyn - ly, ez = lzn - lz;
  // side plane normal s_i = e_i x u_e,i
  const G sx = ey * ez_u - ez * ey_u, sy = ez * ex_u - ex * ez_u, sz = ex * ey_u - ey * ex_u;
  const G spx = __shfl_sync(GVOF_FULL, sx, prv), spy = __shfl_sync(GVOF_FULL, sy, prv),
          spz = __shfl_sync(GVOF_FULL, sz, prv);
  const G dx = spy * sz - spz * sy, dy = spz * sx - spx * sz, dz = spx * sy - spy * sx;
  const G ns = sqrt(sx * sx + sy * sy + sz * sz), nsp = __shfl_sync(GVOF_FULL, ns, prv);
  const G ne = sqrt(ex * ex + ey * ey + ez * ez);
  const G nue = sqrt(ex_u * ex_u + ey_u * ey_u + ez_u * ez_u);
  const G nep = __shfl_sync(GVOF_FULL, ne, prv), nuep = __shfl_sync(GVOF_FULL, nue, prv);
  const G dd = dx * dx + dy * dy + dz * dz;
  // below sin(angle) = 1e-3 the side plane or the line is ill-conditioned
  // (relative error eps/sin) and the streak-line point is used instead
  const G tol = (G)1e-3;
  const bool ok = ns > tol * ne * nue && nsp > tol * nep * nuep && sqrt(dd) > tol * nsp * ns;
  G bxl, byl, bzl;
  if (ok) {
    const G kk = (ux * dx + uy * dy + uz * dz) / dd;
    bxl = lx - kk * dx; byl = ly - kk * dy; bzl = lz - kk * dz;
  } else {
    bxl = lx - ux; byl = ly - uy; bzl = lz - uz;
  }
  fr.degenerate = __popc(__ballot_sync(GVOF_FULL, act && !ok));
  // centroid of the back-traced loop and its vector area B
  const G bxn = __shfl_sync(GVOF_FULL, bxl, nxt), byn = __shfl_sync(GVOF_FULL, byl, nxt),
          bzn = __shfl_sync(GVOF_FULL, bzl, nxt);
  const G xcx = wsum(act ? bxl : G(0)) / (G)I, xcy = wsum(act ? byl : G(0)) / (G)I,
          xcz = wsum(act ? bzl : G(0)) / (G)I;
  const G Bx = wsum(act ? G(0.5) * (byl * bzn - bzl * byn) : G(0));
  const G By = wsum(act ? G(0.5) * (bzl * bxn - bxl * bzn) : G(0));
  const G Bz = wsum(act ? G(0.5) * (bxl * byn - byl * bxn) : G(0));
  // signed volume with the apex at the centroid (origin = face centroid)
  auto det3 = [](G ax, G ay, G az, G bx, G by, G bz, G cx, G cy, G cz) {
    return ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
  };
  G v6 = G(0);
  const G l0x = __shfl_sync(GVOF_FULL, lx, 0), l0y = __shfl_sync(GVOF_FULL, ly, 0),
          l0z = __shfl_sync(GVOF_FULL, lz, 0);
  if (act) {
    if (lane >= 1 && lane + 1 < I) v6 += det3(l0x, l0y, l0z, lx, ly, lz, lxn, lyn, lzn);
    // side quad (x_{i+1}, x_i, b_i, b_{i+1})
    v6 += det3(lxn, lyn, lzn, lx, ly, lz, bxl, byl, bzl);
    v6 += det3(lxn, lyn, lzn, bxl, byl, bzl, bxn, byn, bzn);
    // bottom triangle (b_{i+1}, b_i, apex)
    v6 += det3(bxn, byn, bzn, bxl, byl, bzl, xcx, xcy, xcz);
  }
  const double V0 = wsum((double)v6) / 6.0;
  const double Vl = Vd * fr.sc * fr.sc * fr.sc;
  const double nB = nxd * (double)Bx + nyd * (double)By + nzd * (double)Bz;
  double lam = 0.0;
  fr.edgeon = 0;
  if (fabs(nB) > 1e-8) lam = 3.0 * (V0 - Vl) / nB;
  else fr.edgeon = 1;
  if (act) {
    P.bx[lane] = lx; P.by[lane] = ly; P.bz[lane] = lz;
    P.bx[I + lane] = bxl; P.by[I + lane] = byl; P.bz[I + lane] = bzl;
  }
  if (lane == 0) {
    P.bx[2 * I] = xcx + (G)(lam * nxd);
    P.by[2 * I] = xcy + (G)(lam * nyd);
    P.bz[2 * I] = xcz + (G)(lam * nzd);
  }
  __syncwarp();
  // absolute bounding box
  const int nvb = 2 * I + 1;
  double lo0 = 1e300, lo1 = 1e300, lo2 = 1e300, hi0 = -1e300, hi1 = -1e300, hi2 = -1e300;
  if (lane < nvb) {
    const double ax = fr.cx + fr.L * (double)P.bx[lane];
    const double ay = fr.cy + fr.L * (double)P.by[lane];
    const double az = fr.cz + fr.L * (double)P.bz[lane];
    lo0 = hi0 = ax; lo1 = hi1 = ay; lo2 = hi2 = az;
  }
  // widen by a relative margin so that FP32 rounding never drops a cell
  const double mg = (sizeof(G) == 4 ? 1e-5 : 1e-12) * fr.L;
  fr.lo[0] = wmin(lo0) - mg; fr.lo[1] = wmin(lo1) - mg; fr.lo[2] = wmin(lo2) - mg;
  fr.hi[0] = wmax(hi0) + mg; fr.hi[1] = wmax(hi1) + mg; fr.hi[2] = wmax(hi2) + mg;
  return true;
}

__device__ __forceinline__ bool bbox_overlap(const DevMesh& M, int k, const FaceFrame& fr) {
  const int64_t nc = M.nc;
  return fr.hi[0] > M.bb[k] && fr.lo[0] < M.bb[3 * nc + k] && fr.hi[1] > M.bb[nc + k] &&
         fr.lo[1] < M.bb[4 * nc + k] && fr.hi[2] > M.bb[2 * nc + k] && fr.lo[2] < M.bb[5 * nc + k];
}

__device__ __forceinline__ bool sorted_contains(const int32_t* a, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return lo < n && a[lo] == key;
}

// candidate cells of face j: owner, neighbour and their node neighbours
// (ascending, unique), optionally filtered by tag and bounding box.
// Returns the count written to list (capacity cap), and the full count.
__device__ int candidates(const DevMesh& M, int j, const int8_t* tc, const FaceFrame* fr,
                          int32_t* list, int cap, int lane, int* full) {
  const int own = M.own[j], nbr = M.nbr[j];
  int n = 0;
  const int64_t a0 = M.nb_ptr[own];
  const int na = (int)(M.nb_ptr[own + 1] - a0);
  for (int pass = 0; pass < 2; ++pass) {
    int c0 = pass == 0 ? own : nbr;
    if (c0 < 0) break;
    const int64_t b0 = M.nb_ptr[c0];
    const int nb = (int)(M.nb_ptr[c0 + 1] - b0) + 1;
    for (int base = 0; base < nb; base += 32) {
      const int idx = base + lane;
      int k = -1;
      if (idx < nb) k = (idx == nb - 1) ? c0 : M.nb[b0 + idx];
      bool keep = k >= 0;
      if (keep && pass == 1) keep = !(k == own || sorted_contains(M.nb + a0, na, k));
      if (keep && fr) keep = tc[k] != -1 && bbox_overlap(M, k, *fr);
      const unsigned bal = __ballot_sync(GVOF_FULL, keep);
      if (keep) {
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        if (pos < cap) list[pos] = k;
      }
      n += __popc(bal);
    }
  }
  *full = n;
  const int m = n < cap ? n : cap;
  __syncwarp();
  // rank sort of the distinct entries
  int e[4], r[4];
  for (int q = 0; q < 4; ++q) {
    const int idx = lane + 32 * q;
    e[q] = idx < m ? list[idx] : 0;
    r[q] = 0;
  }
  for (int t = 0; t < m; ++t) {
    const int v = list[t];
    for (int q = 0; q < 4; ++q) r[q] += (v < e[q]);
  }
  __syncwarp();
  for (int q = 0; q < 4; ++q)
    if (lane + 32 * q < m) list[r[q]] = e[q];
  __syncwarp();
  return m;
}

template <typename G>
__global__ void __launch_bounds__(kWarps * 32) k_flux(DevMesh M, DevState S, FluxParams p) {
  __shared__ Poly<G> polys[kWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Poly<G>& P = polys[wib];
  const unsigned n_af = (unsigned)S.cnt[kNAfaces];
  unsigned long long n_trunc = 0, n_over = 0, n_deg = 0, n_edge = 0;
  for (unsigned w = blockIdx.x * kWarps + wib; w < n_af; w += gridDim.x * kWarps) {
    const int j = S.afaces[w];
    const double Vd = S.Vd[j];
    FaceFrame fr;
    if (!build_fmfpa<G>(M, p, j, Vd, P, fr, lane)) {
      if (lane == 0) S.VF[j] = 0.0;
      ++n_over;
      continue;
    }
    n_deg += fr.degenerate;
    n_edge += fr.edgeon;
    int full = 0;
    const int nc = candidates(M, j, S.tc, &fr, P.cand, NCAND, lane, &full);
    unsigned err = 0u;
    if (full > NCAND) err |= 1u;
    double vf = 0.0;
    for (int q = 0; q < nc; ++q) {
      const int k = P.cand[q];
      const int8_t tk = S.tc[k];
      // inward half-spaces of cell k in the face-local frame:
      // -n_out.(x - p_g) >= 0  ->  a = -n_out, b = -n_out.(c - p_g) / L
      const int64_t c0 = M.cf_ptr[k];
      const int nfk = (int)(M.cf_ptr[k + 1] - c0);
      G pa0 = G(0), pa1 = G(0), pa2 = G(0), pb = G(0);
      if (lane < nfk) {
        const int fs = M.cf[c0 + lane];
        const int f = fs >= 0 ? fs : ~fs;
        const double sg = fs >= 0 ? 1.0 : -1.0;
        const double ox = sg * M.fnx[f], oy = sg * M.fny[f], oz = sg * M.fnz[f];
        pa0 = (G)(-ox); pa1 = (G)(-oy); pa2 = (G)(-oz);
        pb = (G)(-(ox * (fr.cx - M.fcx[f]) + oy * (fr.cy - M.fcy[f]) + oz * (fr.cz - M.fcz[f])) * fr.sc);
      }
      PolyState st;
      restore_base(P, st, fr.I, lane);
      int res = 0;
      for (int g = 0; g < nfk && res != 2; ++g) {
        const G a0 = __shfl_sync(GVOF_FULL, pa0, g), a1 = __shfl_sync(GVOF_FULL, pa1, g),
                a2 = __shfl_sync(GVOF_FULL, pa2, g), b = __shfl_sync(GVOF_FULL, pb, g);
        res = clip(P, st, a0, a1, a2, b, lane, err);
      }
      if (res != 2 && tk == 0) {
        // fluid half-space of the PLIC plane: n.(x - x_k) + C >= 0
        const double nx = S.nx[k], ny = S.ny[k], nz = S.nz[k];
        const double b = (nx * (fr.cx - M.ccx[k]) + ny * (fr.cy - M.ccy[k]) + nz * (fr.cz - M.ccz[k]) +
                          S.C[k]) * fr.sc;
        res = clip(P, st, (G)nx, (G)ny, (G)nz, (G)b, lane, err);
      }
      ++n_trunc;
      if (res != 2) vf += volume(P, st, lane);
    }
    if (err) ++n_over;
    if (lane == 0) S.VF[j] = vf * fr.L * fr.L * fr.L;
  }
  if (lane == 0) {
    if (n_trunc) atomicAdd(S.cnt + kNTrunc, n_trunc);
    if (n_over) atomicAdd(S.cnt + kNOverflow, n_over);
    if (n_deg) atomicAdd(S.cnt + kNDegen, n_deg);
    if (n_edge) atomicAdd(S.cnt + kNEdgeOn, n_edge);
  }
}

// export of candidate lists (parity of the overlap lists)
__global__ void k_candidates(DevMesh M, const int32_t* faces, int n, int64_t cap, int32_t* out,
                             int32_t* counts) {
  __shared__ int32_t lists[kWarps][256];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int w = blockIdx.x * kWarps + wib; w < n; w += gridDim.x * kWarps) {
    int full = 0;
    const int m = candidates(M, faces[w], nullptr, nullptr, lists[wib], 128, lane, &full);
    if (lane == 0) counts[w] = full;
    for (int q = lane; q < m && q < cap; q += 32) out[w * cap + q] = lists[wib][q];
    __syncwarp();
  }
}

template <typename G>
__global__ void k_polyhedra(DevMesh M, FluxParams p, const double* srate, const int32_t* faces,
                            int n, double* verts, int32_t* counts) {
  __shared__ Poly<G> polys[kWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Poly<G>& P = polys[wib];
  for (int w = blockIdx.x * kWarps + wib; w < n; w += gridDim.x * kWarps) {
    const int j = faces[w];
    FaceFrame fr;
    const double Vd = srate[j] * p.g * p.dt;
    const bool ok = build_fmfpa<G>(M, p, j, Vd, P, fr, lane);
    if (lane == 0) counts[w] = ok ? fr.I : -1;
    if (ok && lane < 2 * fr.I + 1) {
      verts[(w * NB + lane) * 3 + 0] = fr.cx + fr.L * (double)P.bx[lane];
      verts[(w * NB + lane) * 3 + 1] = fr.cy + fr.L * (double)P.by[lane];
      verts[(w * NB + lane) * 3 + 2] = fr.cz + fr.L * (double)P.bz[lane];
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_flux(const vof_ctx* c, const Vel& v, double g_half, double dt, cudaStream_t s) {
  FluxParams p{v, g_half, dt};
  const int grid = kSMs * 8;
  if (c->opt.precision == VOF_PREC_MIXED)
    k_flux<float><<<grid, kWarps * 32, 0, s>>>(mesh_view(c), state_view(c), p);
  else
    k_flux<double><<<grid, kWarps * 32, 0, s>>>(mesh_view(c), state_view(c), p);
  return cudaGetLastError();
}

cudaError_t launch_candidates(const vof_ctx* c, const int32_t* faces, int n, int64_t cap,
                              int32_t* out, int32_t* counts, cudaStream_t s) {
  k_candidates<<<kSMs, kWarps * 32, 0, s>>>(mesh_view(c), faces, n, cap, out, counts);
  return cudaGetLastError();
}

cudaError_t launch_polyhedra(const vof_ctx* c, const Vel& v, double g_half, double dt,
                             const int32_t* faces, int n, double* verts, int32_t* counts,
                             cudaStream_t s) {
  FluxParams p{v, g_half, dt};
  if (c->opt.precision == VOF_PREC_MIXED)
    k_polyhedra<float><<<kSMs, kWarps * 32, 0, s>>>(mesh_view(c), p, c->srate, faces, n, verts, counts);
  else
    k_polyhedra<double><<<kSMs, kWarps * 32, 0, s>>>(mesh_view(c), p, c->srate, faces, n, verts, counts);
  return cudaGetLastError();
}

}  // namespace gvof

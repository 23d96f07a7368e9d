// PLIC reconstruction of the interfacial cells: LSGIR normal (Sec. 2.1.1,
// Eqs. eq:lsgir1, eq:lsgir2, lsgir-beta) and the volume-enforcing plane
// constant (Sec. 2.1, Eq. plic-eq). One warp per interfacial cell.
//
// Plane constant, GPU design: V(C) = vol(cell ∩ {n.x + C >= 0}) is evaluated
// by clipping each face of the cell (Sutherland-Hodgman) and summing the
// divergence-theorem fan with the origin placed ON the cutting plane, so the
// cap polygon contributes nothing and is never built. Lane v evaluates V at
// the breakpoint C_v = -n.x_v of vertex v; warp max/min reductions give the
// bracket between consecutive breakpoints, where V is exactly a cubic in C.
// Two more evaluations inside the bracket fix the cubic, whose root is found
// by safeguarded Newton iteration.
#include "vof_common.cuh"

namespace gvof {
namespace {

constexpr int kWarps = 4;
constexpr int kMaxCellFaces = 32;
constexpr int kMaxCellVerts = 32;
constexpr int kMaxCellEntries = 128;

struct ReconSmem {
  double x[kMaxCellEntries], y[kMaxCellEntries], z[kMaxCellEntries];  // face loops, cell-local
  int fs[kMaxCellFaces + 1];
};

template <typename G>
__device__ __forceinline__ G warp_sum(G v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(GVOF_FULL, v, o);
  return v;
}

// volume of the part of the cell where n.x + C >= 0 (scaled cell-local frame)
template <typename G>
__device__ G cut_volume(const ReconSmem& S, int nfc, G nx, G ny, G nz, G C) {
  const G ox = -C * nx, oy = -C * ny, oz = -C * nz;  // a point of the plane
  G vol = G(0);
  for (int f = 0; f < nfc; ++f) {
    const int b = S.fs[f], L = S.fs[f + 1] - b;
    G ax = (G)S.x[b + L - 1] - ox, ay = (G)S.y[b + L - 1] - oy, az = (G)S.z[b + L - 1] - oz;
    G pa = nx * ax + ny * ay + nz * az;
    int ne = 0;
    G q0x = 0, q0y = 0, q0z = 0, qpx = 0, qpy = 0, qpz = 0;
    auto emit = [&](G px, G py, G pz) {
      if (ne == 0) { q0x = px; q0y = py; q0z = pz; }
      else if (ne >= 2) {
        vol += q0x * (qpy * pz - qpz * py) + q0y * (qpz * px - qpx * pz) + q0z * (qpx * py - qpy * px);
      }
      qpx = px; qpy = py; qpz = pz;
      ++ne;
    };
    for (int k = 0; k < L; ++k) {
      G bx = (G)S.x[b + k] - ox, by = (G)S.y[b + k] - oy, bz = (G)S.z[b + k] - oz;
      G pb = nx * bx + ny * by + nz * bz;
      bool ia = pa >= G(0), ib = pb >= G(0);
      if (ia != ib) {
        G t = pa / (pa - pb);
        emit(ax + t * (bx - ax), ay + t * (by - ay), az + t * (bz - az));
      }
      if (ib) emit(bx, by, bz);
      ax = bx; ay = by; az = bz; pa = pb;
    }
  }
  return vol / G(6);
}

// plane constant (cell-local, scaled) for target volume T; lanes < ncv hold
// the projection s = n.x_v of vertex v
template <typename G>
__device__ double plane_constant(const ReconSmem& S, int nfc, int ncv, double s_lane, double nxd,
                                 double nyd, double nzd, double Td, int lane) {
  const G nx = (G)nxd, ny = (G)nyd, nz = (G)nzd, T = (G)Td;
  bool has = lane < ncv;
  G Cv = has ? (G)(-s_lane) : G(0);
  G Vv = has ? cut_volume<G>(S, nfc, nx, ny, nz, Cv) : G(0);
  // bracket [Ca, Cb]: largest breakpoint with V <= T, smallest with V >= T
  G Ca = (has && Vv <= T) ? Cv : G(-1e30), Va = Vv;
  G Cb = (has && Vv >= T) ? Cv : G(1e30), Vb = Vv;
  for (int o = 16; o > 0; o >>= 1) {
    G c2 = __shfl_xor_sync(GVOF_FULL, Ca, o), v2 = __shfl_xor_sync(GVOF_FULL, Va, o);
    if (c2 > Ca) { Ca = c2; Va = v2; }
    G c3 = __shfl_xor_sync(GVOF_FULL, Cb, o), v3 = __shfl_xor_sync(GVOF_FULL, Vb, o);
    if (c3 < Cb) { Cb = c3; Vb = v3; }
  }
  if (Va == T || !(Cb > Ca)) return (double)Ca;
  if (Vb == T) return (double)Cb;
  // V is a cubic on [Ca, Cb]: sample at 1/3 and 2/3
  G Cm = Ca + (Cb - Ca) * (G)(lane == 0 ? 1.0 / 3.0 : 2.0 / 3.0);
  G Vm = (lane < 2) ? cut_volume<G>(S, nfc, nx, ny, nz, Cm) : G(0);
  double y0 = (double)Va, y3 = (double)Vb;
  double y1 = (double)__shfl_sync(GVOF_FULL, Vm, 0), y2 = (double)__shfl_sync(GVOF_FULL, Vm, 1);
  // Newton forward form in s = 3 (C - Ca) / (Cb - Ca) in [0, 3]
  double d1 = y1 - y0, d2 = y2 - 2.0 * y1 + y0, d3 = y3 - 3.0 * y2 + 3.0 * y1 - y0;
  double target = (double)Td;
  double lo = 0.0, hi = 3.0;
  double s = 3.0 * (target - y0) / (y3 - y0);
  for (int it = 0; it < 60; ++it) {
    double p = y0 + s * (d1 + (s - 1.0) * (0.5 * d2 + (s - 2.0) * d3 / 6.0));
    double dp = d1 + d2 * (s - 0.5) + d3 * (3.0 * s * s - 6.0 * s + 2.0) / 6.0;
    if (p < target) lo = s; else hi = s;
    double sn = (dp > 0.0) ? s - (p - target) / dp : 0.5 * (lo + hi);
    if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    if (fabs(sn - s) <= 1e-15 * 3.0) { s = sn; break; }
    s = sn;
  }
  return (double)Ca + (s / 3.0) * ((double)Cb - (double)Ca);
}

template <typename G, bool kMixed>
__global__ void __launch_bounds__(kWarps * 32) k_reconstruct(DevMesh M, DevState S, double beta) {
  __shared__ ReconSmem smem[kWarps];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  ReconSmem& Sm = smem[wib];
  const unsigned n_ic = (unsigned)S.cnt[kNIcells];
  for (unsigned w = blockIdx.x * kWarps + wib; w < n_ic; w += gridDim.x * kWarps) {
    const int c = S.icells[w];
    const double xc = M.ccx[c], yc = M.ccy[c], zc = M.ccz[c];
    const double V = M.cvol[c];
    const double hc = cbrt(V), sc = 1.0 / hc;
    const double Fc = S.F[c];
    // ---- LSGIR: weighted least squares for grad F (Sec. 2.1.1)
    G m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0, r0 = 0, r1 = 0, r2 = 0;
    const int64_t q0 = M.nb_ptr[c], q1 = M.nb_ptr[c + 1];
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const int k = M.nb[q];
      G dx = (G)((M.ccx[k] - xc) * sc), dy = (G)((M.ccy[k] - yc) * sc), dz = (G)((M.ccz[k] - zc) * sc);
      G d2 = dx * dx + dy * dy + dz * dz;
      G w2 = (beta == 1.5) ? G(1) / (d2 * sqrt(d2)) : (G)pow((double)d2, -beta);  // w_k^2
      G df = (G)(S.F[k] - Fc);
      m00 += w2 * dx * dx; m01 += w2 * dx * dy; m02 += w2 * dx * dz;
      m11 += w2 * dy * dy; m12 += w2 * dy * dz; m22 += w2 * dz * dz;
      r0 += w2 * dx * df; r1 += w2 * dy * df; r2 += w2 * dz * df;
    }
    m00 = warp_sum(m00); m01 = warp_sum(m01); m02 = warp_sum(m02);
    m11 = warp_sum(m11); m12 = warp_sum(m12); m22 = warp_sum(m22);
    r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2);
    // (A^T A) g = A^T b by the adjugate (symmetric 3x3)
    G a00 = m11 * m22 - m12 * m12, a01 = m02 * m12 - m01 * m22, a02 = m01 * m12 - m02 * m11;
    G a11 = m00 * m22 - m02 * m02, a12 = m01 * m02 - m00 * m12, a22 = m00 * m11 - m01 * m01;
    G det = m00 * a00 + m01 * a01 + m02 * a02;
    G tr = m00 + m11 + m22;
    G gx, gy, gz;
    if (fabs(det) > G(1e-12) * tr * tr * tr) {
      gx = (a00 * r0 + a01 * r1 + a02 * r2);
      gy = (a01 * r0 + a11 * r1 + a12 * r2);
      gz = (a02 * r0 + a12 * r1 + a22 * r2);
      if (det < 0) { gx = -gx; gy = -gy; gz = -gz; }
    } else {
      gx = 1; gy = 0; gz = 0;
    }
    G gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (!(gn > G(0))) { gx = 1; gy = 0; gz = 0; gn = 1; }
    const double nx = (double)(gx / gn), ny = (double)(gy / gn), nz = (double)(gz / gn);

    // ---- cell faces into shared memory (outward loops, cell-local coords)
    const int64_t f0 = M.cf_ptr[c];
    const int nfc = (int)(M.cf_ptr[c + 1] - f0);
    int fid = 0, len = 0;
    bool out = true;
    if (lane < nfc) {
      int fs = M.cf[f0 + lane];
      out = fs >= 0;
      fid = out ? fs : ~fs;
      len = (int)(M.fptr[fid + 1] - M.fptr[fid]);
    }
    int off = len;
    for (int d = 1; d < 32; d <<= 1) {
      int t = __shfl_up_sync(GVOF_FULL, off, d);
      if (lane >= d) off += t;
    }
    if (lane < nfc) {
      Sm.fs[lane + 1] = off;
      off -= len;
      if (lane == 0) Sm.fs[0] = 0;
      const int64_t b = M.fptr[fid];
      for (int i = 0; i < len; ++i) {
        int v = M.fvert[b + (out ? i : len - 1 - i)];
        Sm.x[off + i] = (M.x[v] - xc) * sc;
        Sm.y[off + i] = (M.y[v] - yc) * sc;
        Sm.z[off + i] = (M.z[v] - zc) * sc;
      }
    }
    const int64_t v0 = M.cv_ptr[c];
    const int ncv = (int)(M.cv_ptr[c + 1] - v0);
    double s_lane = 0.0;
    if (lane < ncv) {
      int v = M.cv[v0 + lane];
      s_lane = nx * (M.x[v] - xc) * sc + ny * (M.y[v] - yc) * sc + nz * (M.z[v] - zc) * sc;
    }
    __syncwarp();
    const double T = Fc * V * sc * sc * sc;
    double Cl;
    if (kMixed && (Fc < 1e-3 || Fc > 1.0 - 1e-3))
      Cl = plane_constant<double>(Sm, nfc, ncv, s_lane, nx, ny, nz, T, lane);
    else
      Cl = plane_constant<G>(Sm, nfc, ncv, s_lane, nx, ny, nz, T, lane);
    if (lane == 0) {
      S.nx[c] = nx; S.ny[c] = ny; S.nz[c] = nz;
      S.C[c] = Cl * hc;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_reconstruct(const vof_ctx* c, cudaStream_t s) {
  const int grid = kSMs * 8;
  if (c->opt.precision == VOF_PREC_MIXED)
    k_reconstruct<float, true><<<grid, kWarps * 32, 0, s>>>(mesh_view(c), state_view(c), c->opt.beta);
  else
    k_reconstruct<double, false><<<grid, kWarps * 32, 0, s>>>(mesh_view(c), state_view(c), c->opt.beta);
  return cudaGetLastError();
}

}  // namespace gvof

// Initial volume fraction by refinement (initfgrid, Sec. 3.2), on the device.
//
// The fluid is the part of each cell where the piecewise-linear interpolant
// of the body's signed distance is negative. A cell is the signed sum of the
// tetrahedra (r, p0, a, e) joining its vertex average r to the fan triangles
// (face vertex average p0, edge a-e) of its faces; each tetrahedron is cut
// into ndiv^3 equal pieces (Freudenthal: with w0 = v1 - v0, w1 = v2 - v1,
// w2 = v3 - v2 and lattice coordinates ndiv >= x1 >= x2 >= x3 >= 0 for the
// point v0 + (x1 w0 + x2 w1 + x3 w2) / ndiv, the pieces are the Kuhn
// tetrahedra of the unit lattice cubes inside that simplex). Cells whose
// bounding ball about the centroid lies on one side of the body are 0 or 1.
//
// GPU design: one thread per cell classifies it and lists the cells the
// surface may cross; one warp per listed cell then walks its tetrahedra. The
// classification bounds the range of the distance over a cell (or a
// tetrahedron) about its value at the centre by the body's own geometry,
// tighter than the bounding ball: the largest offset from the centre for a
// sphere, its part across the axis for a cylinder (a slab cell of a quasi-2D
// grid is long along the axis), its part along the normal for a half-space.
// A cell or tetrahedron on one side has the same sign at every lattice
// point, so its fraction is exactly 0 or 1 as the refinement would give. Otherwise the lanes evaluate
// the distance once per lattice point into shared memory (286 points for
// ndiv = 10, against 4000 piece vertices), then share the pieces; a piece
// whose four values agree in sign is 0 or 1, and only the cut ones form
// their fraction, in lattice coordinates (it is affine-invariant; the
// pieces have unit determinant).
// FP64 throughout (the result is an input of both precision paths).
#include "vof_common.cuh"

namespace gvof {
namespace {

constexpr int kWarps = 4;
constexpr int kMaxDiv = 16;
constexpr int kLattice = (kMaxDiv + 1) * (kMaxDiv + 2) * (kMaxDiv + 3) / 6;

struct Shape {
  int kind;
  double cx, cy, cz, ax, ay, az, r;
};

// signed distance to the body, negative inside
__device__ __forceinline__ double shape_phi(const Shape& b, double x, double y, double z) {
  const double dx = x - b.cx, dy = y - b.cy, dz = z - b.cz;
  if (b.kind == VOF_SHAPE_SPHERE) return sqrt(dx * dx + dy * dy + dz * dz) - b.r;
  if (b.kind == VOF_SHAPE_CYLINDER) {
    const double t = dx * b.ax + dy * b.ay + dz * b.az;
    const double px = dx - t * b.ax, py = dy - t * b.ay, pz = dz - t * b.az;
    return sqrt(px * px + py * py + pz * pz) - b.r;
  }
  return b.ax * dx + b.ay * dy + b.az * dz;
}

// how far the distance can move from its value at a point when the point
// moves by d: |d| for a sphere, d across the axis for a cylinder, d along the
// normal for a half-space (each exact for its body)
__device__ __forceinline__ double shape_spread(const Shape& b, double dx, double dy, double dz) {
  if (b.kind == VOF_SHAPE_SPHERE) return sqrt(dx * dx + dy * dy + dz * dz);
  const double t = dx * b.ax + dy * b.ay + dz * b.az;
  if (b.kind == VOF_SHAPE_CYLINDER) {
    const double px = dx - t * b.ax, py = dy - t * b.ay, pz = dz - t * b.az;
    return sqrt(px * px + py * py + pz * pz);
  }
  return fabs(t);
}

__device__ __forceinline__ int lattice_index(int x1, int x2, int x3) {
  return x1 * (x1 + 1) * (x1 + 2) / 6 + x2 * (x2 + 1) / 2 + x3;
}

__device__ __forceinline__ double det3(const double* a, const double* b, const double* c,
                                       const double* d) {
  const double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
  const double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
  const double w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
  return u0 * (v1 * w2 - v2 * w1) - u1 * (v0 * w2 - v2 * w0) + u2 * (v0 * w1 - v1 * w0);
}

// fraction of a piece on the side s > 0 of the linear interpolant of its
// vertex values s (vertices P in lattice coordinates, |det| = 1)
__device__ double piece_fraction(const double P[4][3], const double s[4]) {
  int in[4], ni = 0, out[4], no = 0;
  for (int i = 0; i < 4; ++i) {
    if (s[i] > 0) in[ni++] = i; else out[no++] = i;
  }
  if (ni == 0) return 0.0;
  if (ni == 4) return 1.0;
  if (ni == 1) {
    const int p = in[0];
    double f = 1.0;
    for (int k = 0; k < 3; ++k) f *= s[p] / (s[p] - s[out[k]]);
    return f;
  }
  if (ni == 3) {
    const int o = out[0];
    double f = 1.0;
    for (int k = 0; k < 3; ++k) f *= (-s[o]) / (s[in[k]] - s[o]);
    return 1.0 - f;
  }
  // two on each side: the positive part is the prism (p1, e11, e12 | p2,
  // e21, e22), three tetrahedra
  const int p1 = in[0], p2 = in[1], q1 = out[0], q2 = out[1];
  double a[3][3], b[3][3];
  for (int d = 0; d < 3; ++d) { a[0][d] = P[p1][d]; b[0][d] = P[p2][d]; }
  double t = s[p1] / (s[p1] - s[q1]);
  for (int d = 0; d < 3; ++d) a[1][d] = P[p1][d] + t * (P[q1][d] - P[p1][d]);
  t = s[p1] / (s[p1] - s[q2]);
  for (int d = 0; d < 3; ++d) a[2][d] = P[p1][d] + t * (P[q2][d] - P[p1][d]);
  t = s[p2] / (s[p2] - s[q1]);
  for (int d = 0; d < 3; ++d) b[1][d] = P[p2][d] + t * (P[q1][d] - P[p2][d]);
  t = s[p2] / (s[p2] - s[q2]);
  for (int d = 0; d < 3; ++d) b[2][d] = P[p2][d] + t * (P[q2][d] - P[p2][d]);
  const double v = fabs(det3(a[0], a[1], a[2], b[0])) + fabs(det3(a[1], a[2], b[0], b[1])) +
                   fabs(det3(a[2], b[0], b[1], b[2]));
  return v / fabs(det3(P[0], P[1], P[2], P[3]));
}

// ball test: F = 0 or 1 where the surface cannot cross the cell, else the
// cell goes to the list
__global__ void k_init_classify(DevMesh M, DevState S, Shape b, int32_t* list,
                                unsigned long long* nlist) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < M.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double xc = M.ccx[c], yc = M.ccy[c], zc = M.ccz[c];
    double R = 0.0;
    for (int64_t q = M.cv_ptr[c]; q < M.cv_ptr[c + 1]; ++q) {
      const int v = M.cv[q];
      R = fmax(R, shape_spread(b, M.x[v] - xc, M.y[v] - yc, M.z[v] - zc));
    }
    const double pc = shape_phi(b, xc, yc, zc);
    if (pc > R) {
      S.F[c] = 0.0;
    } else if (pc < -R) {
      S.F[c] = 1.0;
    } else {
      const unsigned long long k = atomicAdd(nlist, 1ull);
      list[k] = (int32_t)c;
    }
  }
}

__global__ void __launch_bounds__(kWarps * 32) k_init_refine(DevMesh M, DevState S, Shape b, int ndiv,
                                                          const int32_t* list,
                                                          const unsigned long long* nlist) {
  __shared__ double lat[kWarps][kLattice];
  // the ndiv^3 pieces of a tetrahedron: base (a1, a2, a3) and step order,
  // packed 4 + 4 + 4 + 3 bits, enumerated once per block
  __shared__ uint16_t pieces[kMaxDiv * kMaxDiv * kMaxDiv];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double* phi = lat[wib];
  if (threadIdx.x == 0) {
    int np = 0;
    for (int a1 = 0; a1 < ndiv; ++a1)
      for (int a2 = 0; a2 <= a1; ++a2)
        for (int a3 = 0; a3 <= a2; ++a3)
          for (int pi = 0; pi < 6; ++pi) {
            const int s0 = pi >> 1, r0 = pi & 1;
            const int s1 = s0 == 0 ? (r0 ? 2 : 1) : (s0 == 1 ? (r0 ? 2 : 0) : (r0 ? 1 : 0));
            const int s2 = 3 - s0 - s1;
            int pos[3];
            pos[s0] = 0; pos[s1] = 1; pos[s2] = 2;
            // where two base coordinates tie, the lower index steps first
            if ((a1 == a2 && pos[0] > pos[1]) || (a2 == a3 && pos[1] > pos[2])) continue;
            pieces[np++] = (uint16_t)(a1 | (a2 << 4) | (a3 << 8) | (pi << 12));
          }
  }
  __syncthreads();
  const int npieces = ndiv * ndiv * ndiv;
  const unsigned n = (unsigned)*nlist;
  const double inv = 1.0 / ndiv;
  for (unsigned w = blockIdx.x * kWarps + wib; w < n; w += gridDim.x * kWarps) {
    const int c = list[w];
    // vertex average of the cell
    double rx = 0, ry = 0, rz = 0;
    const int64_t v0 = M.cv_ptr[c], v1 = M.cv_ptr[c + 1];
    for (int64_t q = v0 + lane; q < v1; q += 32) {
      const int v = M.cv[q];
      rx += M.x[v]; ry += M.y[v]; rz += M.z[v];
    }
    for (int o = 16; o > 0; o >>= 1) {
      rx += __shfl_xor_sync(GVOF_FULL, rx, o);
      ry += __shfl_xor_sync(GVOF_FULL, ry, o);
      rz += __shfl_xor_sync(GVOF_FULL, rz, o);
    }
    const double ncv = (double)(v1 - v0);
    const double r[3] = {rx / ncv, ry / ncv, rz / ncv};
    double vol = 0.0;  // this lane's share of the fluid volume
    for (int64_t q = M.cf_ptr[c]; q < M.cf_ptr[c + 1]; ++q) {
      const int fs = M.cf[q];
      const bool out = fs >= 0;
      const int f = out ? fs : ~fs;
      const int64_t fb = M.fptr[f];
      const int I = (int)(M.fptr[f + 1] - fb);
      double p0[3] = {0, 0, 0};
      for (int i = 0; i < I; ++i) {
        const int v = M.fvert[fb + i];
        p0[0] += M.x[v]; p0[1] += M.y[v]; p0[2] += M.z[v];
      }
      for (int d = 0; d < 3; ++d) p0[d] /= I;
      for (int i = 0; i < I; ++i) {
        const int va = M.fvert[fb + i], ve = M.fvert[fb + (i + 1 == I ? 0 : i + 1)];
        const double A[3] = {M.x[va], M.y[va], M.z[va]}, E[3] = {M.x[ve], M.y[ve], M.z[ve]};
        double T[4][3];
        for (int d = 0; d < 3; ++d) {
          T[0][d] = r[d]; T[1][d] = p0[d];
          T[2][d] = out ? A[d] : E[d];
          T[3][d] = out ? E[d] : A[d];
        }
        const double v = det3(T[0], T[1], T[2], T[3]) / 6.0;
        if (v == 0.0) continue;
        {
          double tc[3], Rt = 0.0;
          for (int d = 0; d < 3; ++d) tc[d] = 0.25 * (T[0][d] + T[1][d] + T[2][d] + T[3][d]);
          for (int k = 0; k < 4; ++k)
            Rt = fmax(Rt, shape_spread(b, T[k][0] - tc[0], T[k][1] - tc[1], T[k][2] - tc[2]));
          const double pt = shape_phi(b, tc[0], tc[1], tc[2]);
          if (pt > Rt) continue;              // no fluid in this tetrahedron
          if (pt < -Rt) {                     // all fluid
            if (lane == 0) vol += v;
            continue;
          }
        }
        double wv[3][3];
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 3; ++d) wv[k][d] = T[k + 1][d] - T[k][d];
        // the body's value at every lattice point (negated: fluid > 0)
        int cnt = 0;
        for (int x1 = 0; x1 <= ndiv; ++x1)
          for (int x2 = 0; x2 <= x1; ++x2)
            for (int x3 = 0; x3 <= x2; ++x3, ++cnt) {
              if ((cnt & 31) != lane) continue;
              double X[3];
              for (int d = 0; d < 3; ++d)
                X[d] = T[0][d] + (x1 * wv[0][d] + x2 * wv[1][d] + x3 * wv[2][d]) * inv;
              phi[lattice_index(x1, x2, x3)] = -shape_phi(b, X[0], X[1], X[2]);
            }
        __syncwarp();
        // the pieces: Kuhn tetrahedra of the lattice cubes at base (a1, a2,
        // a3), a1 >= a2 >= a3, whose steps keep x1 >= x2 >= x3
        double frac = 0.0;
        for (int p = lane; p < npieces; p += 32) {
          const int code = pieces[p];
          const int pi = code >> 12;
          const int s0 = pi >> 1, r0 = pi & 1;
          const int s1 = s0 == 0 ? (r0 ? 2 : 1) : (s0 == 1 ? (r0 ? 2 : 0) : (r0 ? 1 : 0));
          const int s2 = 3 - s0 - s1;
          int x[3] = {code & 15, (code >> 4) & 15, (code >> 8) & 15};
          int xs[4][3];
          double sv[4];
          int npos = 0;
          for (int k = 0; k < 4; ++k) {
            if (k == 1) ++x[s0];
            if (k == 2) ++x[s1];
            if (k == 3) ++x[s2];
            xs[k][0] = x[0]; xs[k][1] = x[1]; xs[k][2] = x[2];
            sv[k] = phi[lattice_index(x[0], x[1], x[2])];
            npos += sv[k] > 0.0;
          }
          if (npos == 0) continue;
          if (npos == 4) { frac += 1.0; continue; }
          double P[4][3];
          for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) P[k][d] = xs[k][d];
          frac += piece_fraction(P, sv);
        }
        vol += v * frac * (inv * inv * inv);
        __syncwarp();
      }
    }
    for (int o = 16; o > 0; o >>= 1) vol += __shfl_xor_sync(GVOF_FULL, vol, o);
    if (lane == 0) {
      const double Fc = vol / M.cvol[c];
      S.F[c] = Fc < 0.0 ? 0.0 : (Fc > 1.0 ? 1.0 : Fc);
    }
  }
}

}  // namespace

cudaError_t launch_init_fraction(const vof_ctx* c, const vof_shape* shape, int ndiv, cudaStream_t s) {
  Shape b;
  b.kind = shape->kind;
  b.cx = shape->c[0]; b.cy = shape->c[1]; b.cz = shape->c[2];
  b.ax = shape->a[0]; b.ay = shape->a[1]; b.az = shape->a[2];
  b.r = shape->r;
  unsigned long long* nlist = c->cnt + kNInitList;
  cudaError_t e = cudaMemsetAsync(nlist, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  // the interfacial-cell list is scratch here: the reconstruction that must
  // follow rebuilds it
  k_init_classify<<<kSMs * 8, 256, 0, s>>>(mesh_view(c), state_view(c), b, c->icells, nlist);
  k_init_refine<<<kSMs * 8, kWarps * 32, 0, s>>>(mesh_view(c), state_view(c), b, ndiv, c->icells, nlist);
  return cudaGetLastError();
}

}  // namespace gvof

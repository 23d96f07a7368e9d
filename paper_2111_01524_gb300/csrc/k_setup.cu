// Set-up kernels: face and cell geometry (the compgrid routine of Sec. 3.1)
// and the per-face flux rate of a separable velocity field.
#include "vof_common.cuh"

namespace gvof {
namespace {

// face vector area, unit normal (out of the owner), area and area centroid
// from the fan of triangles about the vertex average
__global__ void k_face_geometry(DevMesh M, double* fcx, double* fcy, double* fcz, double* fnx,
                                double* fny, double* fnz, double* fa) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < M.nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = M.fptr[f];
    int I = (int)(M.fptr[f + 1] - b);
    double px = 0, py = 0, pz = 0;
    for (int i = 0; i < I; ++i) {
      int v = M.fvert[b + i];
      px += M.x[v]; py += M.y[v]; pz += M.z[v];
    }
    px /= I; py /= I; pz /= I;
    double Ax = 0, Ay = 0, Az = 0;
    for (int i = 0; i < I; ++i) {
      int va = M.fvert[b + i], vb = M.fvert[b + (i + 1 == I ? 0 : i + 1)];
      double ax = M.x[va] - px, ay = M.y[va] - py, az = M.z[va] - pz;
      double bx = M.x[vb] - px, by = M.y[vb] - py, bz = M.z[vb] - pz;
      Ax += 0.5 * (ay * bz - az * by);
      Ay += 0.5 * (az * bx - ax * bz);
      Az += 0.5 * (ax * by - ay * bx);
    }
    double A = sqrt(Ax * Ax + Ay * Ay + Az * Az);
    double nx = Ax / A, ny = Ay / A, nz = Az / A;
    double cx = 0, cy = 0, cz = 0, ws = 0;
    for (int i = 0; i < I; ++i) {
      int va = M.fvert[b + i], vb = M.fvert[b + (i + 1 == I ? 0 : i + 1)];
      double ax = M.x[va] - px, ay = M.y[va] - py, az = M.z[va] - pz;
      double bx = M.x[vb] - px, by = M.y[vb] - py, bz = M.z[vb] - pz;
      double w = 0.5 * (nx * (ay * bz - az * by) + ny * (az * bx - ax * bz) + nz * (ax * by - ay * bx));
      ws += w;
      cx += w * (ax + bx) / 3.0;
      cy += w * (ay + by) / 3.0;
      cz += w * (az + bz) / 3.0;
    }
    fcx[f] = px + cx / ws; fcy[f] = py + cy / ws; fcz[f] = pz + cz / ws;
    fnx[f] = nx; fny[f] = ny; fnz[f] = nz;
    fa[f] = A;
  }
}

// cell volume and centroid from signed tetrahedra (vertex average, face
// vertex average, edge), bounding box, and a convexity flag
__global__ void k_cell_geometry(DevMesh M, double* ccx, double* ccy, double* ccz, double* cvol,
                                double* bb, uint8_t* convex) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < M.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t v0 = M.cv_ptr[c], v1 = M.cv_ptr[c + 1];
    double rx = 0, ry = 0, rz = 0;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t q = v0; q < v1; ++q) {
      int v = M.cv[q];
      double p[3] = {M.x[v], M.y[v], M.z[v]};
      rx += p[0]; ry += p[1]; rz += p[2];
      for (int d = 0; d < 3; ++d) {
        lo[d] = fmin(lo[d], p[d]);
        hi[d] = fmax(hi[d], p[d]);
      }
    }
    double nvc = (double)(v1 - v0);
    rx /= nvc; ry /= nvc; rz /= nvc;
    double vol = 0, mx = 0, my = 0, mz = 0;
    for (int64_t q = M.cf_ptr[c]; q < M.cf_ptr[c + 1]; ++q) {
      int fs = M.cf[q];
      bool out = fs >= 0;
      int f = out ? fs : ~fs;
      int64_t b = M.fptr[f];
      int I = (int)(M.fptr[f + 1] - b);
      double px = 0, py = 0, pz = 0;
      for (int i = 0; i < I; ++i) {
        int v = M.fvert[b + i];
        px += M.x[v]; py += M.y[v]; pz += M.z[v];
      }
      px = px / I - rx; py = py / I - ry; pz = pz / I - rz;
      for (int i = 0; i < I; ++i) {
        int va = M.fvert[b + i], vb = M.fvert[b + (i + 1 == I ? 0 : i + 1)];
        if (!out) { int t = va; va = vb; vb = t; }
        double ax = M.x[va] - rx, ay = M.y[va] - ry, az = M.z[va] - rz;
        double bx = M.x[vb] - rx, by = M.y[vb] - ry, bz = M.z[vb] - rz;
        double v6 = px * (ay * bz - az * by) + py * (az * bx - ax * bz) + pz * (ax * by - ay * bx);
        double v = v6 / 6.0;
        vol += v;
        mx += v * (px + ax + bx) * 0.25;
        my += v * (py + ay + by) * 0.25;
        mz += v * (pz + az + bz) * 0.25;
      }
    }
    cvol[c] = vol;
    ccx[c] = rx + mx / vol; ccy[c] = ry + my / vol; ccz[c] = rz + mz / vol;
    for (int d = 0; d < 3; ++d) {
      bb[d * M.nc + c] = lo[d];
      bb[(3 + d) * M.nc + c] = hi[d];
    }
    // convex: no vertex lies outside the plane of any of its faces; 2: convex
    // and every face normal along an axis (a box: its bounding box is itself)
    double h = cbrt(fabs(vol));
    uint8_t cvx = 1;
    bool axes = true;
    for (int64_t q = M.cf_ptr[c]; q < M.cf_ptr[c + 1] && cvx; ++q) {
      int fs = M.cf[q];
      int f = fs >= 0 ? fs : ~fs;
      double s = fs >= 0 ? 1.0 : -1.0;
      // face centroid is not yet available here; use its first vertex
      int va = M.fvert[M.fptr[f]];
      double nx = 0, ny = 0, nz = 0;
      {
        int64_t b = M.fptr[f];
        int I = (int)(M.fptr[f + 1] - b);
        for (int i = 0; i < I; ++i) {
          int p = M.fvert[b + i], r = M.fvert[b + (i + 1 == I ? 0 : i + 1)];
          nx += M.y[p] * M.z[r] - M.z[p] * M.y[r];
          ny += M.z[p] * M.x[r] - M.x[p] * M.z[r];
          nz += M.x[p] * M.y[r] - M.y[p] * M.x[r];
        }
        double l = sqrt(nx * nx + ny * ny + nz * nz);
        nx /= l; ny /= l; nz /= l;
        const int small = (fabs(nx) < 1e-12) + (fabs(ny) < 1e-12) + (fabs(nz) < 1e-12);
        axes = axes && small == 2;
      }
      for (int64_t p = v0; p < v1; ++p) {
        int v = M.cv[p];
        double d = s * ((M.x[v] - M.x[va]) * nx + (M.y[v] - M.y[va]) * ny + (M.z[v] - M.z[va]) * nz);
        if (d > 1e-10 * h) { cvx = 0; break; }
      }
    }
    convex[c] = cvx && axes ? 2 : cvx;
  }
}

// flux rate (u0(x_f).n_f) A_f of every face and max |u0| per axis over the
// face centres of each grid (for Eq. eq:cfl); the velocity of a face is the
// one of its grid
// radius of a ball about each node inside the union of its cells (the
// node's star): the distance from the node to the nearest plane of a fan
// triangle (face vertex average, edge) of a face of those cells that does
// not contain the node, times 0.999. Faces through the node are shared by
// two cells of the star, so the star's boundary is made of the others, and
// a distance to a triangle's plane is at most the distance to the triangle.
// A node on a boundary face gets 0 (its star does not surround it).
__global__ void k_node_star(DevMesh M, float* rstar) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < M.nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double x = M.x[v], y = M.y[v], z = M.z[v];
    double r = 1e300;
    bool boundary = false;
    for (int64_t q = M.vc_ptr[v]; q < M.vc_ptr[v + 1] && !boundary; ++q) {
      const int c = M.vc[q];
      for (int64_t e = M.cf_ptr[c]; e < M.cf_ptr[c + 1]; ++e) {
        const int fs = M.cf[e];
        const int f = fs >= 0 ? fs : ~fs;
        const int64_t b = M.fptr[f];
        const int I = (int)(M.fptr[f + 1] - b);
        bool has = false;
        for (int i = 0; i < I; ++i) has |= M.fvert[b + i] == v;
        if (has) {
          if (M.nbr[f] < 0) { boundary = true; break; }
          continue;
        }
        double px = 0, py = 0, pz = 0;
        for (int i = 0; i < I; ++i) {
          const int a = M.fvert[b + i];
          px += M.x[a]; py += M.y[a]; pz += M.z[a];
        }
        px /= I; py /= I; pz /= I;
        for (int i = 0; i < I; ++i) {
          const int a = M.fvert[b + i], bb = M.fvert[b + (i + 1 == I ? 0 : i + 1)];
          const double ax = M.x[a] - px, ay = M.y[a] - py, az = M.z[a] - pz;
          const double bx = M.x[bb] - px, by = M.y[bb] - py, bz = M.z[bb] - pz;
          const double nx = ay * bz - az * by, ny = az * bx - ax * bz, nz = ax * by - ay * bx;
          const double nn = sqrt(nx * nx + ny * ny + nz * nz);
          if (nn > 0.0) r = fmin(r, fabs(nx * (x - px) + ny * (y - py) + nz * (z - pz)) / nn);
        }
      }
    }
    rstar[v] = boundary || !(r < 1e300) ? 0.0f : (float)(0.999 * r);
  }
}

__global__ void k_velocity_setup(DevMesh M, const GridParam* gp, double* srate,
                                 unsigned long long* umax) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < M.nf; base += stride) {
    const int64_t f = base + threadIdx.x;
    const bool in = f < M.nf;
    const int g = grid_of(M.face_off, M.n_grids, in ? f : M.nf - 1);
    double m[3] = {0.0, 0.0, 0.0};
    if (in) {
      double u, w, s;
      vel0<double>(gp[g].vel, M.fcx[f], M.fcy[f], M.fcz[f], u, w, s);
      srate[f] = (u * M.fnx[f] + w * M.fny[f] + s * M.fnz[f]) * M.fa[f];
      m[0] = fabs(u); m[1] = fabs(w); m[2] = fabs(s);
    }
    // non-negative doubles order like their bit patterns; one atomic per
    // warp when the warp lies in one grid
    const int g0 = __shfl_sync(GVOF_FULL, g, 0);
    if (__all_sync(GVOF_FULL, g == g0)) {
      for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) m[d] = fmax(m[d], __shfl_xor_sync(GVOF_FULL, m[d], o));
      if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d)
          atomicMax(umax + 3 * g + d, (unsigned long long)__double_as_longlong(m[d]));
    } else if (in) {
      for (int d = 0; d < 3; ++d)
        atomicMax(umax + 3 * g + d, (unsigned long long)__double_as_longlong(m[d]));
    }
  }
}

__device__ __forceinline__ float2 split(double x) {
  float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// (hi, lo) float pairs of the absolute positions and FP32 copies of the
// directions, areas and volumes used by the mixed-precision band kernels
__global__ void k_mixed_copies(DevMesh M, float2* vx2, float2* vy2, float2* vz2, float2* fcx2,
                               float2* fcy2, float2* fcz2, float* fnx32, float* fny32,
                               float* fnz32, float* fa32, float2* ccx2, float2* ccy2,
                               float2* ccz2, float2* bb2, float* cvol32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t v = t0; v < M.nv; v += stride) {
    vx2[v] = split(M.x[v]); vy2[v] = split(M.y[v]); vz2[v] = split(M.z[v]);
  }
  for (int64_t f = t0; f < M.nf; f += stride) {
    fcx2[f] = split(M.fcx[f]); fcy2[f] = split(M.fcy[f]); fcz2[f] = split(M.fcz[f]);
    fnx32[f] = (float)M.fnx[f]; fny32[f] = (float)M.fny[f]; fnz32[f] = (float)M.fnz[f];
    fa32[f] = (float)M.fa[f];
  }
  for (int64_t c = t0; c < M.nc; c += stride) {
    ccx2[c] = split(M.ccx[c]); ccy2[c] = split(M.ccy[c]); ccz2[c] = split(M.ccz[c]);
    cvol32[c] = (float)M.cvol[c];
    for (int d = 0; d < 6; ++d) bb2[6 * c + d] = split(M.bb[d * M.nc + c]);  // one record per cell
  }
}

// per cell face entry: inward unit normal and its offset from the centroid
__global__ void k_cell_planes(DevMesh M, float4* cpl) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < M.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t q = M.cf_ptr[c]; q < M.cf_ptr[c + 1]; ++q) {
      const int fs = M.cf[q];
      const int f = fs >= 0 ? fs : ~fs;
      const double s = fs >= 0 ? -1.0 : 1.0;  // inward = -(outward of this cell)
      const double nx = s * M.fnx[f], ny = s * M.fny[f], nz = s * M.fnz[f];
      const double d = nx * (M.fcx[f] - M.ccx[c]) + ny * (M.fcy[f] - M.ccy[c]) + nz * (M.fcz[f] - M.ccz[c]);
      cpl[q] = make_float4((float)nx, (float)ny, (float)nz, (float)d);
    }
  }
}

inline int grid_for(int64_t n, int bs) {
  int64_t g = (n + bs - 1) / bs;
  int64_t cap = (int64_t)kSMs * 16;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_face_geometry(const vof_ctx* c, cudaStream_t s) {
  k_face_geometry<<<grid_for(c->nf, 256), 256, 0, s>>>(mesh_view(c), c->fcx, c->fcy, c->fcz,
                                                       c->fnx, c->fny, c->fnz, c->fa);
  return cudaGetLastError();
}

cudaError_t launch_cell_geometry(const vof_ctx* c, cudaStream_t s) {
  k_cell_geometry<<<grid_for(c->nc, 256), 256, 0, s>>>(mesh_view(c), c->ccx, c->ccy, c->ccz,
                                                       c->cvol, c->bb, c->convex);
  return cudaGetLastError();
}

cudaError_t launch_node_star(const vof_ctx* c, cudaStream_t s) {
  k_node_star<<<kSMs * 8, 256, 0, s>>>(mesh_view(c), c->rstar);
  return cudaGetLastError();
}

cudaError_t launch_mixed_copies(const vof_ctx* c, cudaStream_t s) {
  int64_t n = c->nf > c->nv ? c->nf : c->nv;
  if (c->nc > n) n = c->nc;
  k_mixed_copies<<<grid_for(n, 256), 256, 0, s>>>(mesh_view(c), c->vx2, c->vy2, c->vz2, c->fcx2,
                                                 c->fcy2, c->fcz2, c->fnx32, c->fny32, c->fnz32,
                                                 c->fa32, c->ccx2, c->ccy2, c->ccz2, c->bb2,
                                                 c->cvol32);
  k_cell_planes<<<grid_for(c->nc, 256), 256, 0, s>>>(mesh_view(c), c->cpl32);
  return cudaGetLastError();
}

cudaError_t launch_velocity_setup(const vof_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->umax_d, 0, 3 * sizeof(unsigned long long) * c->n_grids, s);
  if (e != cudaSuccess) return e;
  k_velocity_setup<<<grid_for(c->nf, 256), 256, 0, s>>>(mesh_view(c), c->gp_d, c->srate, c->umax_d);
  return cudaGetLastError();
}

}  // namespace gvof

/*
 * Oracle for the unsplit geometric VOF step (LSGIR / LSFIR + FMFPA / EMFPA / NMFPA) -- TEST
 * INFRASTRUCTURE ONLY: called by tests/, the smoke check and the CPU-baseline
 * timing; never by the product path. Plain FP64 C, written from the paper
 * (arXiv 2111.01524): Sec. 2.1 (cut-off, PLIC, volume enforcement), Sec.
 * 2.1.1 (LSGIR), Sec. 2.1.2 (LSFIR), Sec. 2.2 (flux volumes, Eq. fnext,
 * clip), Sec. 2.2.1 (EMFPA), Sec. 2.2.2 (FMFPA), Sec. 2.2.3 (NMFPA), Sec. 3 (grid, taggrid), Sec. 4.2 (Eq. eq:cfl, velocity fields).
 *
 * Numerics are deliberately simple and independent of the CUDA library:
 *   - every volume is a sum of signed tetrahedra;
 *   - a tetrahedron is clipped by a plane into 0, 1 or 3 tetrahedra and the
 *     clipping recurses over the planes (no polygon clipping anywhere);
 *   - the plane constant is found by bisection on the cut volume;
 *   - the 3x3 LSGIR system is solved by Gaussian elimination with pivoting.
 *
 * Readings of the paper taken where it is silent: IDW weights
 * 1/|x_node - x_cell|; the cell "geometric
 * centre" is the volume centroid; back-traced FMFPA vertices are the
 * orthogonal projection of the streak-line point onto the side-plane
 * intersection line; the apex of the bottom triangulation moves along the
 * face normal by the closed-form amount that makes the signed volume V_d
 * (both constructions); the EMFPA side-face centre is the vertex average;
 * overlap candidates are the owner, the neighbour and their node neighbours;
 * face tag 1 carries V_F = V_d and face tag -1 carries V_F = 0.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct orc_mesh {
  int64_t nv, nf, nc;
  double* X;
  int64_t* fptr;
  int32_t* fvert;
  int32_t* own;
  int32_t* nbr;
  int64_t* cf_ptr; /* cell -> faces, ascending face id */
  int32_t* cf;
  int64_t* cv_ptr; /* cell -> vertices, ascending */
  int32_t* cv;
  int64_t* vc_ptr; /* vertex -> cells, ascending */
  int32_t* vc;
  int64_t* nb_ptr; /* neigbcell, ascending, self excluded */
  int32_t* nb;
  double* fc;  /* face area centroid */
  double* fn;  /* unit normal out of the owner */
  double* fa;  /* area */
  double* fp0; /* face vertex average (fan point) */
  double* cc;  /* cell centroid */
  double* cvol;
  double* bbox; /* min xyz, max xyz */
  uint8_t* convex;
};

/* ------------------------------------------------------------- op counter */
/* floating-point operations of the truncations, per thread: each counted
 * routine adds the adds, subtracts, multiplies and divides it performs (a
 * comparison or a sign change is not counted). orc_faceflux reports the sum
 * over its (face, cell) truncations in stats[4]; the count measures the work
 * of this plain algorithm, it does not change any result. */
static _Thread_local int64_t g_flops;
#define ORC_FLOPS(n) (g_flops += (n))

/* ---------------------------------------------------------------- vectors */
static void sub3(const double* a, const double* b, double* r) {
  r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double* a, const double* b, double* r) {
  double x = a[1] * b[2] - a[2] * b[1];
  double y = a[2] * b[0] - a[0] * b[2];
  double z = a[0] * b[1] - a[1] * b[0];
  r[0] = x; r[1] = y; r[2] = z;
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
/* 6 x signed volume of tetrahedron (a, b, c, d) */
static double det6(const double* a, const double* b, const double* c, const double* d) {
  double u[3], v[3], w[3], x[3];
  sub3(b, a, u); sub3(c, a, v); sub3(d, a, w);
  cross3(v, w, x);
  return dot3(u, x);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}
static int64_t sort_unique(int32_t* v, int64_t n) {
  if (n == 0) return 0;
  qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
  int64_t k = 1;
  for (int64_t i = 1; i < n; ++i)
    if (v[i] != v[k - 1]) v[k++] = v[i];
  return k;
}

/* ----------------------------------------------------------- mesh (Sec 3.1) */
orc_mesh* orc_mesh_build(int64_t nv, const double* X, int64_t nf,
                         const int64_t* fptr, const int32_t* fvert,
                         const int32_t* own, const int32_t* nbr, int64_t nc) {
  if (nv <= 0 || nf <= 0 || nc <= 0) return NULL;
  for (int64_t f = 0; f < nf; ++f) {
    if (own[f] < 0 || own[f] >= nc || nbr[f] >= nc) return NULL;
    if (fptr[f + 1] - fptr[f] < 3) return NULL;
  }
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->nv = nv; m->nf = nf; m->nc = nc;
  int64_t nfv = fptr[nf];
  m->X = (double*)malloc(sizeof(double) * 3 * nv);
  memcpy(m->X, X, sizeof(double) * 3 * nv);
  m->fptr = (int64_t*)malloc(sizeof(int64_t) * (nf + 1));
  memcpy(m->fptr, fptr, sizeof(int64_t) * (nf + 1));
  m->fvert = (int32_t*)malloc(sizeof(int32_t) * nfv);
  memcpy(m->fvert, fvert, sizeof(int32_t) * nfv);
  m->own = (int32_t*)malloc(sizeof(int32_t) * nf);
  memcpy(m->own, own, sizeof(int32_t) * nf);
  m->nbr = (int32_t*)malloc(sizeof(int32_t) * nf);
  memcpy(m->nbr, nbr, sizeof(int32_t) * nf);

  /* cell -> faces (faces visited in ascending order, so lists are sorted) */
  m->cf_ptr = (int64_t*)calloc(nc + 1, sizeof(int64_t));
  for (int64_t f = 0; f < nf; ++f) {
    m->cf_ptr[own[f] + 1]++;
    if (nbr[f] >= 0) m->cf_ptr[nbr[f] + 1]++;
  }
  for (int64_t c = 0; c < nc; ++c) m->cf_ptr[c + 1] += m->cf_ptr[c];
  m->cf = (int32_t*)malloc(sizeof(int32_t) * m->cf_ptr[nc]);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * nc);
  memcpy(fill, m->cf_ptr, sizeof(int64_t) * nc);
  for (int64_t f = 0; f < nf; ++f) {
    m->cf[fill[own[f]]++] = (int32_t)f;
    if (nbr[f] >= 0) m->cf[fill[nbr[f]]++] = (int32_t)f;
  }

  /* cell -> vertices (per-cell sorted unique; counted, then filled) */
  m->cv_ptr = (int64_t*)calloc(nc + 1, sizeof(int64_t));
  int64_t* rawp = (int64_t*)calloc(nc + 1, sizeof(int64_t));
  for (int64_t c = 0; c < nc; ++c) {
    int64_t s = 0;
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
      int32_t f = m->cf[q];
      s += fptr[f + 1] - fptr[f];
    }
    rawp[c + 1] = rawp[c] + s;
  }
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (rawp[nc] > 0 ? rawp[nc] : 1));
  int64_t* ucnt = (int64_t*)malloc(sizeof(int64_t) * nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t pos = rawp[c];
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
      int32_t f = m->cf[q];
      for (int64_t k = fptr[f]; k < fptr[f + 1]; ++k) tmp[pos++] = fvert[k];
    }
    ucnt[c] = sort_unique(tmp + rawp[c], rawp[c + 1] - rawp[c]);
  }
  for (int64_t c = 0; c < nc; ++c) m->cv_ptr[c + 1] = m->cv_ptr[c] + ucnt[c];
  int64_t pos = m->cv_ptr[nc];
  m->cv = (int32_t*)malloc(sizeof(int32_t) * (pos > 0 ? pos : 1));
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c)
    memcpy(m->cv + m->cv_ptr[c], tmp + rawp[c], sizeof(int32_t) * ucnt[c]);
  free(tmp);
  free(rawp);

  /* vertex -> cells (cells visited in ascending order) */
  m->vc_ptr = (int64_t*)calloc(nv + 1, sizeof(int64_t));
  for (int64_t q = 0; q < m->cv_ptr[nc]; ++q) m->vc_ptr[m->cv[q] + 1]++;
  for (int64_t v = 0; v < nv; ++v) m->vc_ptr[v + 1] += m->vc_ptr[v];
  m->vc = (int32_t*)malloc(sizeof(int32_t) * (m->vc_ptr[nv] > 0 ? m->vc_ptr[nv] : 1));
  int64_t* vfill = (int64_t*)malloc(sizeof(int64_t) * nv);
  memcpy(vfill, m->vc_ptr, sizeof(int64_t) * nv);
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q)
      m->vc[vfill[m->cv[q]]++] = (int32_t)c;
  free(vfill);

  /* neigbcell: cells sharing at least one node (Sec. 3.1); two passes */
  m->nb_ptr = (int64_t*)calloc(nc + 1, sizeof(int64_t));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      for (int64_t c = 0; c < nc; ++c) m->nb_ptr[c + 1] = m->nb_ptr[c] + ucnt[c];
      m->nb = (int32_t*)malloc(sizeof(int32_t) * (m->nb_ptr[nc] > 0 ? m->nb_ptr[nc] : 1));
    }
#pragma omp parallel
    {
      int64_t cap = 1024;
      int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * cap);
#pragma omp for schedule(dynamic, 1024)
      for (int64_t c = 0; c < nc; ++c) {
        int64_t k = 0;
        for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q) {
          int32_t v = m->cv[q];
          for (int64_t r = m->vc_ptr[v]; r < m->vc_ptr[v + 1]; ++r) {
            if (k == cap) { cap *= 2; buf = (int32_t*)realloc(buf, sizeof(int32_t) * cap); }
            buf[k++] = m->vc[r];
          }
        }
        k = sort_unique(buf, k);
        if (pass == 0) { ucnt[c] = k - 1; continue; }
        int64_t w = m->nb_ptr[c];
        for (int64_t i = 0; i < k; ++i)
          if (buf[i] != c) m->nb[w++] = buf[i];
      }
      free(buf);
    }
  }
  free(ucnt);

  /* face geometry (compgrid) */
  m->fc = (double*)malloc(sizeof(double) * 3 * nf);
  m->fn = (double*)malloc(sizeof(double) * 3 * nf);
  m->fa = (double*)malloc(sizeof(double) * nf);
  m->fp0 = (double*)malloc(sizeof(double) * 3 * nf);
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < nf; ++f) {
    int64_t b = fptr[f], I = fptr[f + 1] - b;
    double p0[3] = {0, 0, 0};
    for (int64_t i = 0; i < I; ++i)
      for (int d = 0; d < 3; ++d) p0[d] += X[3 * fvert[b + i] + d];
    for (int d = 0; d < 3; ++d) p0[d] /= (double)I;
    double A[3] = {0, 0, 0};
    double tri[64][3];
    double tc[64][3];
    int ntri = (int)(I < 64 ? I : 64);
    for (int64_t i = 0; i < ntri; ++i) {
      const double* a = X + 3 * fvert[b + i];
      const double* c = X + 3 * fvert[b + (i + 1) % I];
      double u[3], w[3];
      sub3(a, p0, u); sub3(c, p0, w);
      cross3(u, w, tri[i]);
      for (int d = 0; d < 3; ++d) {
        tri[i][d] *= 0.5;
        A[d] += tri[i][d];
        tc[i][d] = (p0[d] + a[d] + c[d]) / 3.0;
      }
    }
    double area = norm3(A);
    double n[3] = {A[0] / area, A[1] / area, A[2] / area};
    double cen[3] = {0, 0, 0}, wsum = 0;
    for (int i = 0; i < ntri; ++i) {
      double w = dot3(tri[i], n);
      wsum += w;
      for (int d = 0; d < 3; ++d) cen[d] += w * tc[i][d];
    }
    for (int d = 0; d < 3; ++d) {
      m->fc[3 * f + d] = cen[d] / wsum;
      m->fn[3 * f + d] = n[d];
      m->fp0[3 * f + d] = p0[d];
    }
    m->fa[f] = area;
  }

  /* cell geometry: signed tetrahedra from the cell's vertex average over the
   * fan triangles of its faces, oriented outward */
  m->cc = (double*)malloc(sizeof(double) * 3 * nc);
  m->cvol = (double*)malloc(sizeof(double) * nc);
  m->bbox = (double*)malloc(sizeof(double) * 6 * nc);
  m->convex = (uint8_t*)malloc(nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    double r[3] = {0, 0, 0};
    int64_t ncv = m->cv_ptr[c + 1] - m->cv_ptr[c];
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q) {
      const double* x = X + 3 * m->cv[q];
      for (int d = 0; d < 3; ++d) {
        r[d] += x[d];
        if (x[d] < lo[d]) lo[d] = x[d];
        if (x[d] > hi[d]) hi[d] = x[d];
      }
    }
    for (int d = 0; d < 3; ++d) r[d] /= (double)ncv;
    double vol = 0, cen[3] = {0, 0, 0};
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
      int32_t f = m->cf[q];
      int out = (own[f] == c);
      int64_t b = fptr[f], I = fptr[f + 1] - b;
      for (int64_t i = 0; i < I; ++i) {
        const double* a = X + 3 * fvert[b + i];
        const double* e = X + 3 * fvert[b + (i + 1) % I];
        const double* p0 = m->fp0 + 3 * f;
        double v6 = out ? det6(r, p0, a, e) : det6(r, p0, e, a);
        double v = v6 / 6.0;
        vol += v;
        for (int d = 0; d < 3; ++d) cen[d] += v * (r[d] + p0[d] + a[d] + e[d]) / 4.0;
      }
    }
    m->cvol[c] = vol;
    for (int d = 0; d < 3; ++d) {
      m->cc[3 * c + d] = cen[d] / vol;
      m->bbox[6 * c + d] = lo[d];
      m->bbox[6 * c + 3 + d] = hi[d];
    }
    /* convex if every vertex lies on the inner side of every face plane */
    double h = cbrt(fabs(vol));
    int cvx = 1;
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1] && cvx; ++q) {
      int32_t f = m->cf[q];
      double s = (own[f] == c) ? 1.0 : -1.0;
      for (int64_t p = m->cv_ptr[c]; p < m->cv_ptr[c + 1]; ++p) {
        double d[3];
        sub3(X + 3 * m->cv[p], m->fc + 3 * f, d);
        if (s * dot3(d, m->fn + 3 * f) > 1e-10 * h) { cvx = 0; break; }
      }
    }
    m->convex[c] = (uint8_t)cvx;
  }
  free(fill);
  return m;
}

void orc_mesh_free(orc_mesh* m) {
  if (!m) return;
  free(m->X); free(m->fptr); free(m->fvert); free(m->own); free(m->nbr);
  free(m->cf_ptr); free(m->cf); free(m->cv_ptr); free(m->cv);
  free(m->vc_ptr); free(m->vc); free(m->nb_ptr); free(m->nb);
  free(m->fc); free(m->fn); free(m->fa); free(m->fp0);
  free(m->cc); free(m->cvol); free(m->bbox); free(m->convex);
  free(m);
}

void orc_geometry(const orc_mesh* m, double* cell_vol, double* cell_cen,
                  double* face_cen, double* face_nrm, double* face_area,
                  double* cell_bbox, uint8_t* cell_convex) {
  if (cell_vol) memcpy(cell_vol, m->cvol, sizeof(double) * m->nc);
  if (cell_cen) memcpy(cell_cen, m->cc, sizeof(double) * 3 * m->nc);
  if (face_cen) memcpy(face_cen, m->fc, sizeof(double) * 3 * m->nf);
  if (face_nrm) memcpy(face_nrm, m->fn, sizeof(double) * 3 * m->nf);
  if (face_area) memcpy(face_area, m->fa, sizeof(double) * m->nf);
  if (cell_bbox) memcpy(cell_bbox, m->bbox, sizeof(double) * 6 * m->nc);
  if (cell_convex) memcpy(cell_convex, m->convex, (size_t)m->nc);
}

int64_t orc_neighbors(const orc_mesh* m, int64_t* ptr, int32_t* idx) {
  if (ptr) memcpy(ptr, m->nb_ptr, sizeof(int64_t) * (m->nc + 1));
  if (idx) memcpy(idx, m->nb, sizeof(int32_t) * m->nb_ptr[m->nc]);
  return m->nb_ptr[m->nc];
}

int orc_candidates(const orc_mesh* m, int64_t f, int32_t* out, int cap) {
  int32_t cells[2] = {m->own[f], m->nbr[f]};
  int64_t n = 0;
  int64_t need = 2;
  for (int s = 0; s < 2; ++s)
    if (cells[s] >= 0) need += m->nb_ptr[cells[s] + 1] - m->nb_ptr[cells[s]];
  int32_t* t = (int32_t*)malloc(sizeof(int32_t) * need);
  for (int s = 0; s < 2; ++s) {
    int32_t c = cells[s];
    if (c < 0) continue;
    t[n++] = c;
    for (int64_t q = m->nb_ptr[c]; q < m->nb_ptr[c + 1]; ++q) t[n++] = m->nb[q];
  }
  n = sort_unique(t, n);
  int w = (int)(n < cap ? n : cap);
  memcpy(out, t, sizeof(int32_t) * w);
  free(t);
  return (int)n;
}

/* --------------------------------------------------------- taggrid (Sec 3.3) */
void orc_taggrid(const orc_mesh* m, double eps, double* F, double* Fnode,
                 int8_t* tag_v, int8_t* tag_f, int8_t* tag_c) {
  /* cut-off of uniform cells (Sec. 2.1) and cell tags */
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < m->nc; ++c) {
    if (F[c] < eps) { F[c] = 0.0; tag_c[c] = -1; }
    else if (F[c] > 1.0 - eps) { F[c] = 1.0; tag_c[c] = 1; }
    else tag_c[c] = 0;
  }
  /* node values by inverse-distance weighting, node tags */
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < m->nv; ++v) {
    double num = 0, den = 0;
    for (int64_t q = m->vc_ptr[v]; q < m->vc_ptr[v + 1]; ++q) {
      int32_t c = m->vc[q];
      double d[3];
      sub3(m->X + 3 * v, m->cc + 3 * c, d);
      double w = 1.0 / norm3(d);
      num += w * F[c];
      den += w;
    }
    double fs = num / den;
    if (Fnode) Fnode[v] = fs;
    tag_v[v] = (int8_t)(fs < eps ? -1 : (fs > 1.0 - eps ? 1 : 0));
  }
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < m->nf; ++f) {
    int all_m = 1, all_p = 1;
    for (int64_t k = m->fptr[f]; k < m->fptr[f + 1]; ++k) {
      int8_t t = tag_v[m->fvert[k]];
      if (t != -1) all_m = 0;
      if (t != 1) all_p = 0;
    }
    tag_f[f] = (int8_t)(all_m ? -1 : (all_p ? 1 : 0));
  }
}

/* ----------------------------------------------------------- LSGIR (Sec 2.1.1) */
static void sym3_jacobi(double A[3][3], double V[3][3]);
static int solve3(double M[3][3], double r[3], double g[3]) {
  /* Gaussian elimination with partial pivoting */
  int piv[3] = {0, 1, 2};
  double A[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) A[i][j] = M[i][j];
    A[i][3] = r[i];
  }
  (void)piv;
  double scale = fabs(M[0][0]) + fabs(M[1][1]) + fabs(M[2][2]);
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
    if (fabs(A[p][k]) <= 1e-14 * scale) return -1;
    if (p != k)
      for (int j = 0; j < 4; ++j) { double t = A[k][j]; A[k][j] = A[p][j]; A[p][j] = t; }
    for (int i = k + 1; i < 3; ++i) {
      double l = A[i][k] / A[k][k];
      for (int j = k; j < 4; ++j) A[i][j] -= l * A[k][j];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double s = A[i][3];
    for (int j = i + 1; j < 3; ++j) s -= A[i][j] * g[j];
    g[i] = s / A[i][i];
  }
  return 0;
}

void orc_lsgir(const orc_mesh* m, double beta, const double* F,
               const int8_t* tag_c, double* nrm) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t c = 0; c < m->nc; ++c) {
    nrm[3 * c] = nrm[3 * c + 1] = nrm[3 * c + 2] = 0.0;
    if (tag_c[c] != 0) continue;
    double M[3][3] = {{0}}, r[3] = {0, 0, 0};
    for (int64_t q = m->nb_ptr[c]; q < m->nb_ptr[c + 1]; ++q) {
      int32_t k = m->nb[q];
      double d[3];
      sub3(m->cc + 3 * k, m->cc + 3 * c, d);
      double w = pow(norm3(d), -beta); /* Eq. lsgir-beta */
      double w2 = w * w;
      double db = F[k] - F[c];
      for (int i = 0; i < 3; ++i) {
        r[i] += w2 * d[i] * db; /* A^T b */
        for (int j = 0; j < 3; ++j) M[i][j] += w2 * d[i] * d[j]; /* A^T A */
      }
    }
    double g[3];
    if (solve3(M, r, g) != 0) {
      /* singular stencil (e.g. a quasi-2D grid, one cell thick: every
       * neighbour offset lies in the plane): least-squares solution of
       * minimum norm, by the pseudo-inverse over the eigenvalues above
       * 1e-12 of the largest */
      double A[3][3], V[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = M[i][j];
      sym3_jacobi(A, V);
      double top = fmax(A[0][0], fmax(A[1][1], A[2][2]));
      g[0] = g[1] = g[2] = 0.0;
      for (int k = 0; k < 3; ++k) {
        if (!(A[k][k] > 1e-12 * top)) continue;
        double vr = V[0][k] * r[0] + V[1][k] * r[1] + V[2][k] * r[2];
        for (int i = 0; i < 3; ++i) g[i] += vr / A[k][k] * V[i][k];
      }
      if (!(norm3(g) > 0)) { g[0] = 1; g[1] = 0; g[2] = 0; }
    }
    double gn = norm3(g);
    if (!(gn > 0)) { g[0] = 1; g[1] = 0; g[2] = 0; gn = 1; }
    for (int i = 0; i < 3; ++i) nrm[3 * c + i] = g[i] / gn;
  }
}

/* --------------------------------------------- cut volumes and plane constant */
/* fraction of a tetrahedron on the side s > 0 of a plane, from the signed
 * plane values s[4] at its vertices and its vertex coordinates */
static double tet_inside_fraction(const double P[4][3], const double s[4]) {
  int in[4], ni = 0, out[4], no = 0;
  for (int i = 0; i < 4; ++i) {
    if (s[i] > 0) in[ni++] = i; else out[no++] = i;
  }
  if (ni == 0) return 0.0;
  if (ni == 4) return 1.0;
  if (ni == 1) {
    int p = in[0];
    double f = 1.0;
    for (int k = 0; k < 3; ++k) f *= s[p] / (s[p] - s[out[k]]);
    return f;
  }
  if (ni == 3) {
    int o = out[0];
    double f = 1.0;
    for (int k = 0; k < 3; ++k) f *= (-s[o]) / (s[in[k]] - s[o]);
    return 1.0 - f;
  }
  /* two inside: prism (p1, e11, e12 | p2, e21, e22), three tetrahedra */
  double a[3][3], b[3][3];
  int p1 = in[0], p2 = in[1], q1 = out[0], q2 = out[1];
  double t;
  for (int d = 0; d < 3; ++d) { a[0][d] = P[p1][d]; b[0][d] = P[p2][d]; }
  t = s[p1] / (s[p1] - s[q1]);
  for (int d = 0; d < 3; ++d) a[1][d] = P[p1][d] + t * (P[q1][d] - P[p1][d]);
  t = s[p1] / (s[p1] - s[q2]);
  for (int d = 0; d < 3; ++d) a[2][d] = P[p1][d] + t * (P[q2][d] - P[p1][d]);
  t = s[p2] / (s[p2] - s[q1]);
  for (int d = 0; d < 3; ++d) b[1][d] = P[p2][d] + t * (P[q1][d] - P[p2][d]);
  t = s[p2] / (s[p2] - s[q2]);
  for (int d = 0; d < 3; ++d) b[2][d] = P[p2][d] + t * (P[q2][d] - P[p2][d]);
  double v = fabs(det6(a[0], a[1], a[2], b[0])) + fabs(det6(a[1], a[2], b[0], b[1])) +
             fabs(det6(a[2], b[0], b[1], b[2]));
  double vt = fabs(det6(P[0], P[1], P[2], P[3]));
  return v / vt;
}

/* vol(cell ∩ {n.(x - xc) + C >= 0}) by signed tetrahedra (Sec. 2.1) */
double orc_cell_cut_volume(const orc_mesh* m, int64_t c, const double n[3], double C) {
  double r[3] = {0, 0, 0};
  int64_t ncv = m->cv_ptr[c + 1] - m->cv_ptr[c];
  for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q)
    for (int d = 0; d < 3; ++d) r[d] += m->X[3 * m->cv[q] + d];
  for (int d = 0; d < 3; ++d) r[d] /= (double)ncv;
  const double* xc = m->cc + 3 * c;
  double vol = 0.0;
  for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
    int32_t f = m->cf[q];
    int out = (m->own[f] == c);
    int64_t b = m->fptr[f], I = m->fptr[f + 1] - b;
    for (int64_t i = 0; i < I; ++i) {
      double P[4][3];
      const double* a = m->X + 3 * m->fvert[b + i];
      const double* e = m->X + 3 * m->fvert[b + (i + 1) % I];
      const double* p0 = m->fp0 + 3 * f;
      for (int d = 0; d < 3; ++d) {
        P[0][d] = r[d]; P[1][d] = p0[d];
        P[2][d] = out ? a[d] : e[d];
        P[3][d] = out ? e[d] : a[d];
      }
      double v = det6(P[0], P[1], P[2], P[3]) / 6.0;
      if (v == 0.0) continue;
      double s[4];
      for (int k = 0; k < 4; ++k) {
        double dd[3];
        sub3(P[k], xc, dd);
        s[k] = dot3(n, dd) + C;
      }
      vol += v * tet_inside_fraction(P, s);
    }
  }
  return vol;
}

void orc_plane_constant(const orc_mesh* m, const double* F, const int8_t* tag_c,
                        const double* nrm, double* Cout) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t c = 0; c < m->nc; ++c) {
    Cout[c] = 0.0;
    if (tag_c[c] != 0) continue;
    const double* n = nrm + 3 * c;
    const double* xc = m->cc + 3 * c;
    double smin = 1e300, smax = -1e300;
    for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q) {
      double d[3];
      sub3(m->X + 3 * m->cv[q], xc, d);
      double s = dot3(n, d);
      if (s < smin) smin = s;
      if (s > smax) smax = s;
    }
    /* V(-smax) = 0, V(-smin) = V_cell; V is non-decreasing in C */
    double lo = -smax, hi = -smin;
    double target = F[c] * m->cvol[c];
    for (int it = 0; it < 200; ++it) {
      double mid = lo + 0.5 * (hi - lo);
      if (mid <= lo || mid >= hi) break;
      if (orc_cell_cut_volume(m, c, n, mid) < target) lo = mid; else hi = mid;
    }
    Cout[c] = lo + 0.5 * (hi - lo);
  }
}

/* ------------------------------------------------------- initfgrid (Sec 3.2) */
/* implicit function of the initial fluid body: negative inside; a signed
 * distance (1-Lipschitz) for every kind, so that a cell whose bounding ball
 * lies on one side is entirely fluid or empty.
 * kind 1: sphere (centre c, radius r); 2: infinite cylinder (axis through c
 * along the unit vector a, radius r); 3: half-space a.(x - c) < 0 (a unit). */
static double body_phi(const orc_body* b, const double x[3]) {
  double d[3];
  sub3(x, b->c, d);
  if (b->kind == 1) return norm3(d) - b->r;
  if (b->kind == 2) {
    double t = dot3(d, b->a);
    double p[3] = {d[0] - t * b->a[0], d[1] - t * b->a[1], d[2] - t * b->a[2]};
    return norm3(p) - b->r;
  }
  return dot3(b->a, d);
}

/* volume fraction of the fluid (the part of every cell where the piecewise
 * linear interpolant of phi is negative) by refinement: each cell is the
 * signed sum of the tetrahedra joining its vertex average to the fan
 * triangles of its faces; each tetrahedron (v0, v1, v2, v3) is divided into
 * ndiv^3 equal tetrahedra (Freudenthal: in the coordinates x with point
 * v0 + (x1 (v1 - v0) + x2 (v2 - v1) + x3 (v3 - v2)) / ndiv, the simplex is
 * ndiv >= x1 >= x2 >= x3 >= 0, and its pieces are the Kuhn tetrahedra of the
 * unit lattice cubes that lie in it); phi is evaluated at their vertices
 * and the negative part of each piece is exact for the linear interpolant.
 * Cells whose bounding ball about the centroid lies on one side of the body
 * are 0 or 1 without refinement. */
void orc_initfgrid(const orc_mesh* m, const orc_body* body, int ndiv, double* F) {
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t c = 0; c < m->nc; ++c) {
    const double* xc = m->cc + 3 * c;
    double R = 0.0;
    for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q) {
      double d[3];
      sub3(m->X + 3 * m->cv[q], xc, d);
      double l = norm3(d);
      if (l > R) R = l;
    }
    double pc = body_phi(body, xc);
    if (pc > R) { F[c] = 0.0; continue; }
    if (pc < -R) { F[c] = 1.0; continue; }
    double r[3] = {0, 0, 0};
    int64_t ncv = m->cv_ptr[c + 1] - m->cv_ptr[c];
    for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q)
      for (int d = 0; d < 3; ++d) r[d] += m->X[3 * m->cv[q] + d];
    for (int d = 0; d < 3; ++d) r[d] /= (double)ncv;
    double vol = 0.0;
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
      int32_t f = m->cf[q];
      int out = (m->own[f] == c);
      int64_t b = m->fptr[f], I = m->fptr[f + 1] - b;
      const double* p0 = m->fp0 + 3 * f;
      for (int64_t i = 0; i < I; ++i) {
        const double* a = m->X + 3 * m->fvert[b + i];
        const double* e = m->X + 3 * m->fvert[b + (i + 1) % I];
        double T[4][3];
        for (int d = 0; d < 3; ++d) {
          T[0][d] = r[d]; T[1][d] = p0[d];
          T[2][d] = out ? a[d] : e[d];
          T[3][d] = out ? e[d] : a[d];
        }
        double v = det6(T[0], T[1], T[2], T[3]) / 6.0;
        if (v == 0.0) continue;
        double w[3][3]; /* v1 - v0, v2 - v1, v3 - v2 */
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 3; ++d) w[k][d] = T[k + 1][d] - T[k][d];
        double frac = 0.0;
        for (int a1 = 0; a1 < ndiv; ++a1)
          for (int a2 = 0; a2 <= a1; ++a2)
            for (int a3 = 0; a3 <= a2; ++a3) {
              int base[3] = {a1, a2, a3};
              for (int pi = 0; pi < 6; ++pi) {
                const int* pr = perm[pi];
                /* where two base coordinates tie, the lower index steps first */
                int pos[3];
                for (int k = 0; k < 3; ++k) pos[pr[k]] = k;
                if ((a1 == a2 && pos[0] > pos[1]) || (a2 == a3 && pos[1] > pos[2])) continue;
                double S[4][3], sv[4];
                int x[3] = {base[0], base[1], base[2]};
                for (int k = 0; k < 4; ++k) {
                  if (k > 0) x[pr[k - 1]] += 1;
                  for (int d = 0; d < 3; ++d)
                    S[k][d] = T[0][d] + (x[0] * w[0][d] + x[1] * w[1][d] + x[2] * w[2][d]) / ndiv;
                  sv[k] = -body_phi(body, S[k]);
                }
                frac += tet_inside_fraction(S, sv);
              }
            }
        vol += v * frac / ((double)ndiv * ndiv * ndiv);
      }
    }
    double Fc = vol / m->cvol[c];
    F[c] = Fc < 0.0 ? 0.0 : (Fc > 1.0 ? 1.0 : Fc);
  }
}

/* ------------------------------------------------------------ LSFIR (Sec 2.1.2) */
/* geometric centre of the vertex set of the PLIC polygon of cell c, plane
 * n.(x - xc) + C = 0: the points where the plane crosses an edge of the
 * cell (ends strictly on opposite sides), each edge once, and the cell
 * vertices that lie on the plane. Returns the number of points (0: the
 * plane misses the cell; out = the centroid). */
int orc_plic_centre(const orc_mesh* m, int64_t c, const double n[3], double C, double out[3]) {
  const double* xc = m->cc + 3 * c;
  /* the cell's edges, each once as (low id, high id) */
  int32_t ea[256], eb[256];
  int ne = 0;
  for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
    int32_t f = m->cf[q];
    int64_t b = m->fptr[f], I = m->fptr[f + 1] - b;
    for (int64_t i = 0; i < I; ++i) {
      int32_t a = m->fvert[b + i], e = m->fvert[b + (i + 1) % I];
      int32_t lo = a < e ? a : e, hi = a < e ? e : a;
      int seen = 0;
      for (int k = 0; k < ne && !seen; ++k) seen = (ea[k] == lo && eb[k] == hi);
      if (!seen && ne < 256) { ea[ne] = lo; eb[ne] = hi; ++ne; }
    }
  }
  double sum[3] = {0, 0, 0};
  int np = 0;
  for (int k = 0; k < ne; ++k) {
    const double* A = m->X + 3 * ea[k];
    const double* B = m->X + 3 * eb[k];
    double da[3], db[3];
    sub3(A, xc, da);
    sub3(B, xc, db);
    double pa = dot3(n, da) + C, pb = dot3(n, db) + C;
    if ((pa > 0 && pb < 0) || (pa < 0 && pb > 0)) {
      double t = pa / (pa - pb);
      for (int d = 0; d < 3; ++d) sum[d] += A[d] + t * (B[d] - A[d]);
      ++np;
    }
  }
  for (int64_t q = m->cv_ptr[c]; q < m->cv_ptr[c + 1]; ++q) {
    const double* V = m->X + 3 * m->cv[q];
    double dv[3];
    sub3(V, xc, dv);
    if (dot3(n, dv) + C == 0.0) {
      for (int d = 0; d < 3; ++d) sum[d] += V[d];
      ++np;
    }
  }
  if (np == 0) {
    for (int d = 0; d < 3; ++d) out[d] = xc[d];
    return 0;
  }
  for (int d = 0; d < 3; ++d) out[d] = sum[d] / np;
  return np;
}

/* eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
 * (each rotation in the (p, q) plane zeroes A[p][q]); on return the
 * diagonal of A holds the eigenvalues and the columns of V the vectors */
static void sym3_jacobi(double A[3][3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j);
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-32 * dia || off == 0.0) break;
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; ++r) {
      int p = P[r][0], q = P[r][1];
      if (A[p][q] == 0.0) continue;
      /* angle with tan(2 phi) = 2 A_pq / (A_qq - A_pp); the smaller root t */
      double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
      double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
      double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      J[p][p] = cs; J[q][q] = cs; J[p][q] = sn; J[q][p] = -sn;
      double T[3][3], R[3][3];
      /* A <- J^T A J, V <- V J */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          T[i][j] = 0;
          for (int k = 0; k < 3; ++k) T[i][j] += A[i][k] * J[k][j];
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          R[i][j] = 0;
          for (int k = 0; k < 3; ++k) R[i][j] += J[k][i] * T[k][j];
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = R[i][j];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          T[i][j] = 0;
          for (int k = 0; k < 3; ++k) T[i][j] += V[i][k] * J[k][j];
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = T[i][j];
    }
  }
}

/* angle between unit vectors, accurate for small angles */
static double angle3(const double* a, const double* b) {
  double x[3];
  cross3(a, b, x);
  return atan2(norm3(x), dot3(a, b));
}

/* one LSFIR normal update (Sec. 2.1.2): for each interfacial cell, the unit
 * normal of the plane through its PLIC centre x that minimises
 * H = sum_k w_k delta_k^2 over the valid interfacial neighbours k (node
 * neighbours whose previous normal is within 45 degrees of the cell's, the
 * SWIR validity rule of Sec. 2.1.2), delta_k = n.(x_k - x), w_k =
 * |x_k - x|^-2.5: the eigenvector of the smallest eigenvalue of
 * sum_k w_k d_k d_k^T, oriented like the previous normal. A cell with fewer
 * than two valid neighbours, or whose two smallest eigenvalues are equal
 * (collinear centres: no unique plane), keeps its normal. cand receives
 * the normals; returns the number of cells that kept theirs. */
int64_t orc_lsfir_normals(const orc_mesh* m, const int8_t* tag_c, const double* nrm,
                          const double* xp, double* cand) {
  const double cos45 = sqrt(0.5);
  int64_t kept = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : kept)
  for (int64_t c = 0; c < m->nc; ++c) {
    for (int d = 0; d < 3; ++d) cand[3 * c + d] = nrm[3 * c + d];
    if (tag_c[c] != 0) continue;
    const double* nc_ = nrm + 3 * c;
    double M[3][3] = {{0}};
    int nvalid = 0;
    for (int64_t q = m->nb_ptr[c]; q < m->nb_ptr[c + 1]; ++q) {
      int32_t k = m->nb[q];
      if (tag_c[k] != 0) continue;
      if (!(dot3(nc_, nrm + 3 * k) > cos45)) continue;
      double d[3];
      sub3(xp + 3 * k, xp + 3 * c, d);
      double r2 = dot3(d, d);
      if (!(r2 > 0)) continue;
      double w = pow(r2, -1.25); /* |d|^-2.5 */
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] += w * d[i] * d[j];
      ++nvalid;
    }
    if (nvalid < 2) { ++kept; continue; }
    double V[3][3];
    sym3_jacobi(M, V);
    int lo = 0;
    for (int i = 1; i < 3; ++i)
      if (M[i][i] < M[lo][lo]) lo = i;
    int i1 = (lo + 1) % 3, i2 = (lo + 2) % 3;
    double mid = M[i1][i1] < M[i2][i2] ? M[i1][i1] : M[i2][i2];
    double top = M[i1][i1] < M[i2][i2] ? M[i2][i2] : M[i1][i1];
    if (!(mid - M[lo][lo] > 1e-12 * top)) { ++kept; continue; }
    double v[3] = {V[0][lo], V[1][lo], V[2][lo]};
    double vn = norm3(v);
    double sg = dot3(v, nc_) < 0 ? -1.0 : 1.0;
    for (int d = 0; d < 3; ++d) cand[3 * c + d] = sg * v[d] / vn;
  }
  return kept;
}

/* acceptance step of outer iteration io (Sec. 2.1.2): each interfacial
 * cell takes its candidate normal when it turns the current one by less than
 * 30 degrees / io; every cell is decided from the normals before the step.
 * Returns the largest accepted turn (radians). */
double orc_lsfir_accept(const orc_mesh* m, const int8_t* tag_c, int io, const double* cand,
                        double* nrm) {
  const double pi = 3.14159265358979323846;
  const double lim = (30.0 * pi / 180.0) / io;
  double turned = 0.0;
  for (int64_t c = 0; c < m->nc; ++c) {
    if (tag_c[c] != 0) continue;
    double a = angle3(nrm + 3 * c, cand + 3 * c);
    if (a < lim) {
      for (int d = 0; d < 3; ++d) nrm[3 * c + d] = cand[3 * c + d];
      if (a > turned) turned = a;
    }
  }
  return turned;
}

/* LSFIR reconstruction (Sec. 2.1.2) with the outer iteration of Sec. 2.1.2:
 * from the normals given in nrm (the LSGIR ones, Sec. 2.1.1), repeat up to
 * n_out times: PLIC centres of the current planes; candidate normals; each
 * interfacial cell takes its candidate if it turns its normal by less than
 * 30 degrees / I_out (all cells updated together, after every candidate is
 * known); the plane constants are enforced again (Sec. 2.1). Stops after the
 * iteration in which no normal turned by tol or more. C receives the final
 * plane constants. Returns the number of outer iterations done. */
int orc_lsfir(const orc_mesh* m, int n_out, double tol, const double* F, const int8_t* tag_c,
              double* nrm, double* C) {
  double* xp = (double*)malloc(sizeof(double) * 3 * m->nc);
  double* cand = (double*)malloc(sizeof(double) * 3 * m->nc);
  orc_plane_constant(m, F, tag_c, nrm, C);
  int it = 0;
  for (int io = 1; io <= n_out; ++io) {
    it = io;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < m->nc; ++c) {
      if (tag_c[c] == 0) orc_plic_centre(m, c, nrm + 3 * c, C[c], xp + 3 * c);
      else for (int d = 0; d < 3; ++d) xp[3 * c + d] = m->cc[3 * c + d];
    }
    orc_lsfir_normals(m, tag_c, nrm, xp, cand);
    double turned = orc_lsfir_accept(m, tag_c, io, cand, nrm);
    orc_plane_constant(m, F, tag_c, nrm, C);
    if (turned < tol) break;
  }
  free(xp);
  free(cand);
  return it;
}

/* ------------------------------------------------------ velocity (Sec 4.2) */
void orc_velocity_eval(const orc_velocity* v, const double x[3], double t, double u[3]) {
  const double pi = 3.14159265358979323846;
  if (v->kind == 1) { /* 3D deformation (Enright) */
    double g = cos(pi * t / v->period);
    double sx = sin(pi * x[0]), sy = sin(pi * x[1]), sz = sin(pi * x[2]);
    double s2x = sin(2 * pi * x[0]), s2y = sin(2 * pi * x[1]), s2z = sin(2 * pi * x[2]);
    u[0] = 2.0 * sx * sx * s2y * s2z * g;
    u[1] = -s2x * sy * sy * s2z * g;
    u[2] = -s2x * s2y * sz * sz * g;
  } else if (v->kind == 4) { /* 2D deformation in the x-z plane (Sec. 4.3) */
    double g = cos(pi * t / v->period);
    double sx = sin(pi * x[0]), sz = sin(pi * x[2]);
    u[0] = -2.0 * sx * sx * sz * cos(pi * x[2]) * g;
    u[1] = 0.0;
    u[2] = 2.0 * sz * sz * sx * cos(pi * x[0]) * g;
  } else if (v->kind == 2) { /* rigid rotation about a z-parallel axis */
    u[0] = -v->omega * (x[1] - v->center[1]);
    u[1] = v->omega * (x[0] - v->center[0]);
    u[2] = 0.0;
  } else { /* uniform translation */
    u[0] = v->u0[0]; u[1] = v->u0[1]; u[2] = v->u0[2];
  }
}

/* --------------------------------------------------------- FMFPA (Sec 2.2.2) */
static double poly_volume_loops(int nv, const double* V, int nf, const int* fp, const int* fi);

/* face loops of a flux polyhedron over its vertex list (outward orientation
 * for V_d > 0); returns the number of loops.
 * method 0, FMFPA (Sec. 2.2.2): vertices x_0..x_{I-1}, back-traced
 *   x_I..x_{2I-1}, apex 2I; loops: the cell face, I side quads, I bottom
 *   triangles (2I+1 faces).
 * method 1, EMFPA (Sec. 2.2.1): vertices as above, then the side-face
 *   centres s_0..s_{I-1} at 2I..3I-1 and the apex at 3I; each side face
 *   (x_{i+1}, x_i, x_{I+i}, x_{I+i+1}) is replaced by the four triangles
 *   that join its edges to s_i (5I+1 faces).
 * method 2, NMFPA (Sec. 2.2.3): vertices x_0..x_{2I-1} only; loops: the
 *   cell face, I planar side quads, the back-traced face (I+2 faces). */
static int flux_loops(int method, int I, int* fp, int* fi) {
  int nfp = 0, k = 0;
  fp[0] = 0;
  for (int i = 0; i < I; ++i) fi[k++] = i;
  fp[++nfp] = k;
  for (int i = 0; i < I; ++i) {
    int ip = (i + 1) % I;
    int q[4] = {ip, i, I + i, I + ip};
    if (method == 1) {
      for (int e = 0; e < 4; ++e) {
        fi[k++] = q[e]; fi[k++] = q[(e + 1) % 4]; fi[k++] = 2 * I + i;
        fp[++nfp] = k;
      }
    } else {
      for (int e = 0; e < 4; ++e) fi[k++] = q[e];
      fp[++nfp] = k;
    }
  }
  if (method == 2) {
    /* the back-traced face, reversed (its outward normal is -n) */
    for (int i = I - 1; i >= 0; --i) fi[k++] = I + i;
    fp[++nfp] = k;
    return nfp;
  }
  int apex = method == 1 ? 3 * I : 2 * I;
  for (int i = 0; i < I; ++i) {
    int ip = (i + 1) % I;
    fi[k++] = I + ip; fi[k++] = I + i; fi[k++] = apex;
    fp[++nfp] = k;
  }
  return nfp;
}

/* apex of the bottom triangulation: the centroid xc of the back-traced loop
 * xb moved along the face normal n so that the closed surface has signed
 * volume Vd (Sec. 2.2.1). Moving the apex by lam n changes the volume by
 * -lam n.B/3, B the vector area of the back-traced loop, so lam = 3(V0 -
 * Vd)/(n.B) with V0 the volume at lam = 0. Returns 0, or 2 if the loop is
 * edge-on (|n.B| <= 1e-8 A) and the apex stays at xc. */
static int place_apex(int nvp, double (*P)[3], int nfp, const int* fp, const int* fi,
                      double (*xb)[3], int I, const double* n, double A, double Vd,
                      int apex) {
  double xc[3] = {0, 0, 0};
  for (int i = 0; i < I; ++i)
    for (int q = 0; q < 3; ++q) xc[q] += xb[i][q] / I;
  for (int q = 0; q < 3; ++q) P[apex][q] = xc[q];
  double V0 = poly_volume_loops(nvp, &P[0][0], nfp, fp, fi);
  double B[3] = {0, 0, 0};
  for (int i = 0; i < I; ++i) {
    double w[3];
    cross3(xb[i], xb[(i + 1) % I], w);
    for (int q = 0; q < 3; ++q) B[q] += 0.5 * w[q];
  }
  double nB = dot3(n, B);
  double lam = 0.0;
  int fl = 0;
  if (fabs(nB) > 1e-8 * A) lam = 3.0 * (V0 - Vd) / nB;
  else fl = 2;
  for (int q = 0; q < 3; ++q) P[apex][q] = xc[q] + lam * n[q];
  return fl;
}

/* --------------------------------------------------------- EMFPA (Sec 2.2.1) */
int orc_emfpa(const orc_mesh* m, int64_t f, const orc_velocity* vel, double th,
              double dt, double* out, int capI, double* Vd, int* flags) {
  int64_t b = m->fptr[f];
  int I = (int)(m->fptr[f + 1] - b);
  if (I > capI || I > 32) return -1;
  const double* c = m->fc + 3 * f;
  const double* n = m->fn + 3 * f;
  double uc[3];
  orc_velocity_eval(vel, c, th, uc);
  *Vd = dot3(uc, n) * m->fa[f] * dt; /* Eq. a-donacion */
  /* frame with origin at the face centroid; every vertex goes back along
   * its own streak line with the velocity at t^{n+1/2} (Eq. streak-line2) */
  double P[97][3], xb[32][3];
  for (int i = 0; i < I; ++i) {
    const double* xa = m->X + 3 * m->fvert[b + i];
    double u[3];
    orc_velocity_eval(vel, xa, th, u);
    sub3(xa, c, P[i]);
    for (int q = 0; q < 3; ++q) xb[i][q] = P[i][q] - dt * u[q];
  }
  for (int i = 0; i < I; ++i) {
    int ip = (i + 1) % I;
    for (int q = 0; q < 3; ++q) {
      P[I + i][q] = xb[i][q];
      /* geometric centre of side face i: plain vertex average */
      P[2 * I + i][q] = 0.25 * (P[i][q] + P[ip][q] + xb[i][q] + xb[ip][q]);
    }
  }
  int nvp = 3 * I + 1;
  int fp[5 * 32 + 2], fi[16 * 32];
  int nfp = flux_loops(1, I, fp, fi);
  *flags = place_apex(nvp, P, nfp, fp, fi, xb, I, n, m->fa[f], *Vd, 3 * I);
  for (int i = 0; i < nvp; ++i)
    for (int q = 0; q < 3; ++q) out[3 * i + q] = P[i][q] + c[q];
  return I;
}

/* --------------------------------------------------------- NMFPA (Sec 2.2.3) */
/* every vertex of the face goes back with the one velocity of the face
 * centre at t^{n+1/2} (Eq. streak-line2 with u_c): the polyhedron is the
 * prism between the face and its translate, whose volume is V_d itself
 * (no apex, no adjustment) */
int orc_nmfpa(const orc_mesh* m, int64_t f, const orc_velocity* vel, double th,
              double dt, double* out, int capI, double* Vd, int* flags) {
  int64_t b = m->fptr[f];
  int I = (int)(m->fptr[f + 1] - b);
  if (I > capI || I > 32) return -1;
  const double* c = m->fc + 3 * f;
  const double* n = m->fn + 3 * f;
  double uc[3];
  orc_velocity_eval(vel, c, th, uc);
  *Vd = dot3(uc, n) * m->fa[f] * dt; /* Eq. a-donacion */
  *flags = 0;
  for (int i = 0; i < I; ++i) {
    const double* xa = m->X + 3 * m->fvert[b + i];
    double x[3];
    sub3(xa, c, x);
    for (int q = 0; q < 3; ++q) {
      out[3 * i + q] = x[q] + c[q];
      out[3 * (I + i) + q] = (x[q] - dt * uc[q]) + c[q];
    }
  }
  return I;
}

int orc_fmfpa(const orc_mesh* m, int64_t f, const orc_velocity* vel, double th,
              double dt, double* out, int capI, double* Vd, int* flags) {
  int64_t b = m->fptr[f];
  int I = (int)(m->fptr[f + 1] - b);
  if (I > capI || I > 32) return -1;
  const double* c = m->fc + 3 * f;
  const double* n = m->fn + 3 * f;
  double uc[3];
  orc_velocity_eval(vel, c, th, uc);
  *Vd = dot3(uc, n) * m->fa[f] * dt; /* Eq. a-donacion */
  *flags = 0;
  /* local frame: origin at the face centroid */
  double x[32][3], ue[32][3], uv[32][3], s[32][3];
  for (int i = 0; i < I; ++i) {
    const double* xa = m->X + 3 * m->fvert[b + i];
    const double* xb = m->X + 3 * m->fvert[b + (i + 1) % I];
    double mid[3];
    for (int d = 0; d < 3; ++d) mid[d] = 0.5 * (xa[d] + xb[d]);
    orc_velocity_eval(vel, mid, th, ue[i]); /* velocity at the edge centre */
    orc_velocity_eval(vel, xa, th, uv[i]);  /* velocity at the vertex */
    sub3(xa, c, x[i]);
  }
  /* side plane i contains edge i and is parallel to ue[i] */
  for (int i = 0; i < I; ++i) {
    double e[3];
    sub3(x[(i + 1) % I], x[i], e);
    cross3(e, ue[i], s[i]);
  }
  double xb[32][3];
  for (int i = 0; i < I; ++i) {
    int im = (i + I - 1) % I;
    double d[3];
    cross3(s[im], s[i], d);
    double e0[3], e1[3];
    sub3(x[(i + 1) % I], x[i], e0);
    sub3(x[i], x[im], e1);
    /* a side plane is undefined when its edge is (nearly) parallel to the
     * edge-centre velocity, and the line is undefined when the two side
     * planes are (nearly) parallel; the back-traced point then has a
     * relative error of order eps/sin(angle), so below sin = 1e-3 the
     * streak-line point is used instead */
    const double tol = 1e-3;
    int ok_s = norm3(s[i]) > tol * norm3(e0) * norm3(ue[i]) &&
               norm3(s[im]) > tol * norm3(e1) * norm3(ue[im]);
    double dd = dot3(d, d);
    if (ok_s && sqrt(dd) > tol * norm3(s[im]) * norm3(s[i])) {
      /* back-trace along the line of intersection of the two side planes:
       * orthogonal projection of the streak-line displacement on the line */
      double k = dt * dot3(uv[i], d) / dd;
      for (int q = 0; q < 3; ++q) xb[i][q] = x[i][q] - k * d[q];
    } else {
      for (int q = 0; q < 3; ++q) xb[i][q] = x[i][q] - dt * uv[i][q]; /* Eq. streak-line2 */
      *flags |= 1;
    }
  }
  /* polyhedron: x_0..x_{I-1}, xb_0..xb_{I-1}, apex */
  int nvp = 2 * I + 1;
  double P[65][3];
  for (int i = 0; i < I; ++i)
    for (int q = 0; q < 3; ++q) { P[i][q] = x[i][q]; P[I + i][q] = xb[i][q]; }
  int fp[66], fi[66 * 4];
  int nfp = flux_loops(0, I, fp, fi);
  *flags |= place_apex(nvp, P, nfp, fp, fi, xb, I, n, m->fa[f], *Vd, 2 * I);
  for (int i = 0; i < nvp; ++i)
    for (int q = 0; q < 3; ++q) out[3 * i + q] = P[i][q] + c[q];
  return I;
}

/* ------------------------------------------------ truncation by tetrahedra */
/* volume of tetrahedron T clipped by planes[k] (a.x + b > 0), recursively:
 * each plane leaves 0, 1 or 3 tetrahedra */
static double tet_clip(const double T[4][3], const double* planes, int np) {
  if (np == 0) {
    ORC_FLOPS(24);  /* det6 (23) and the division */
    return fabs(det6(T[0], T[1], T[2], T[3])) / 6.0;
  }
  double s[4];
  int in[4], ni = 0, out[4], no = 0;
  ORC_FLOPS(24);  /* four plane values: 3 mul + 3 add each */
  for (int i = 0; i < 4; ++i) {
    s[i] = planes[0] * T[i][0] + planes[1] * T[i][1] + planes[2] * T[i][2] + planes[3];
    if (s[i] > 0) in[ni++] = i; else out[no++] = i;
  }
  if (ni == 0) return 0.0;
  if (ni == 4) return tet_clip(T, planes + 4, np - 1);
  double R[4][3];
  /* each cut point: t (sub, div) and three (sub, mul, add) */
  ORC_FLOPS(ni == 2 ? 4 * 11 : 3 * 11);
  if (ni == 1) {
    int p = in[0];
    for (int d = 0; d < 3; ++d) R[0][d] = T[p][d];
    for (int k = 0; k < 3; ++k) {
      double t = s[p] / (s[p] - s[out[k]]);
      for (int d = 0; d < 3; ++d) R[k + 1][d] = T[p][d] + t * (T[out[k]][d] - T[p][d]);
    }
    return tet_clip(R, planes + 4, np - 1);
  }
  /* prism a0 a1 a2 | b0 b1 b2 with lateral edges a_i - b_i */
  double a[3][3], b[3][3];
  if (ni == 3) {
    int o = out[0];
    for (int k = 0; k < 3; ++k) {
      double t = s[in[k]] / (s[in[k]] - s[o]);
      for (int d = 0; d < 3; ++d) {
        a[k][d] = T[in[k]][d];
        b[k][d] = T[in[k]][d] + t * (T[o][d] - T[in[k]][d]);
      }
    }
  } else {
    int p1 = in[0], p2 = in[1], q1 = out[0], q2 = out[1];
    double t;
    for (int d = 0; d < 3; ++d) { a[0][d] = T[p1][d]; b[0][d] = T[p2][d]; }
    t = s[p1] / (s[p1] - s[q1]);
    for (int d = 0; d < 3; ++d) a[1][d] = T[p1][d] + t * (T[q1][d] - T[p1][d]);
    t = s[p1] / (s[p1] - s[q2]);
    for (int d = 0; d < 3; ++d) a[2][d] = T[p1][d] + t * (T[q2][d] - T[p1][d]);
    t = s[p2] / (s[p2] - s[q1]);
    for (int d = 0; d < 3; ++d) b[1][d] = T[p2][d] + t * (T[q1][d] - T[p2][d]);
    t = s[p2] / (s[p2] - s[q2]);
    for (int d = 0; d < 3; ++d) b[2][d] = T[p2][d] + t * (T[q2][d] - T[p2][d]);
  }
  double v = 0.0;
  for (int d = 0; d < 3; ++d) {
    R[0][d] = a[0][d]; R[1][d] = a[1][d]; R[2][d] = a[2][d]; R[3][d] = b[0][d];
  }
  v += tet_clip(R, planes + 4, np - 1);
  for (int d = 0; d < 3; ++d) {
    R[0][d] = a[1][d]; R[1][d] = a[2][d]; R[2][d] = b[0][d]; R[3][d] = b[1][d];
  }
  v += tet_clip(R, planes + 4, np - 1);
  for (int d = 0; d < 3; ++d) {
    R[0][d] = a[2][d]; R[1][d] = b[0][d]; R[2][d] = b[1][d]; R[3][d] = b[2][d];
  }
  v += tet_clip(R, planes + 4, np - 1);
  return v;
}

/* signed volume of a closed surface given as face loops: fan each loop from
 * its first vertex and sum the tetrahedra (origin, a, b, c) / 6 */
static double poly_volume_loops(int nv, const double* V, int nf, const int* fp, const int* fi) {
  (void)nv;
  double o[3] = {0, 0, 0};
  double vol = 0.0;
  for (int f = 0; f < nf; ++f) {
    int b = fp[f], L = fp[f + 1] - b;
    for (int i = 1; i + 1 < L; ++i)
      vol += det6(o, V + 3 * fi[b], V + 3 * fi[b + i], V + 3 * fi[b + i + 1]) / 6.0;
  }
  return vol;
}

double orc_poly_volume(int nv, const double* V, int nf, const int* fp, const int* fi) {
  return poly_volume_loops(nv, V, nf, fp, fi);
}

/* P ∩ planes: signed tetrahedra (apex = first vertex of P) over the fan
 * triangles of P's faces; each clipped by the planes (winding-number sum) */
double orc_poly_clip_volume(int nv, const double* V, int nf, const int* fp,
                            const int* fi, int np, const double* planes) {
  (void)nv;
  const double* apex = V + 3 * fi[0];
  double vol = 0.0;
  for (int f = 0; f < nf; ++f) {
    int b = fp[f], L = fp[f + 1] - b;
    for (int i = 1; i + 1 < L; ++i) {
      double T[4][3];
      const double* p[4] = {apex, V + 3 * fi[b], V + 3 * fi[b + i], V + 3 * fi[b + i + 1]};
      for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) T[k][d] = p[k][d];
      double d6 = det6(T[0], T[1], T[2], T[3]);
      ORC_FLOPS(23 + 2);  /* det6, the signed sum */
      if (d6 == 0.0) continue;
      double sgn = d6 > 0 ? 1.0 : -1.0;
      vol += sgn * tet_clip(T, planes, np);
    }
  }
  return vol;
}

/* inward half-space of the plane through p with outward normal nout,
 * expressed in the frame with origin o:  -nout.(x + o - p) > 0 */
static void inward_plane(const double* nout, const double* p, const double* o, double* pl) {
  ORC_FLOPS(8);  /* sub3, dot3 */
  pl[0] = -nout[0]; pl[1] = -nout[1]; pl[2] = -nout[2];
  double d[3];
  sub3(o, p, d);
  pl[3] = -dot3(nout, d);
}

/* vol(P ∩ cell k ∩ fluid_k), P given in the frame with origin o */
static double truncate_in_cell(const orc_mesh* m, int nv, const double* V, int nf,
                               const int* fp, const int* fi, int32_t k, int8_t tag,
                               const double* nrm, const double* Cp, const double* o) {
  double planes[4 * 40];
  int np = 0;
  if (m->convex[k]) {
    for (int64_t q = m->cf_ptr[k]; q < m->cf_ptr[k + 1] && np < 38; ++q) {
      int32_t f = m->cf[q];
      double s = (m->own[f] == k) ? 1.0 : -1.0;
      double nout[3] = {s * m->fn[3 * f], s * m->fn[3 * f + 1], s * m->fn[3 * f + 2]};
      inward_plane(nout, m->fc + 3 * f, o, planes + 4 * np);
      ++np;
    }
    if (tag == 0) {
      /* fluid side n.(x - xc) + C > 0 */
      const double* n = nrm + 3 * k;
      double d[3];
      ORC_FLOPS(9);  /* sub3, dot3, add */
      sub3(o, m->cc + 3 * k, d);
      planes[4 * np] = n[0]; planes[4 * np + 1] = n[1]; planes[4 * np + 2] = n[2];
      planes[4 * np + 3] = dot3(n, d) + Cp[k];
      ++np;
    }
    return orc_poly_clip_volume(nv, V, nf, fp, fi, np, planes);
  }
  /* non-convex cell: signed tetrahedra (vertex average, face fan) */
  double r[3] = {0, 0, 0};
  int64_t ncv = m->cv_ptr[k + 1] - m->cv_ptr[k];
  for (int64_t q = m->cv_ptr[k]; q < m->cv_ptr[k + 1]; ++q)
    for (int d = 0; d < 3; ++d) r[d] += m->X[3 * m->cv[q] + d];
  for (int d = 0; d < 3; ++d) r[d] = r[d] / (double)ncv - o[d];
  double vol = 0.0;
  for (int64_t q = m->cf_ptr[k]; q < m->cf_ptr[k + 1]; ++q) {
    int32_t f = m->cf[q];
    int out = (m->own[f] == k);
    int64_t b = m->fptr[f], I = m->fptr[f + 1] - b;
    double p0[3];
    sub3(m->fp0 + 3 * f, o, p0);
    for (int64_t i = 0; i < I; ++i) {
      double A[3], E[3];
      sub3(m->X + 3 * m->fvert[b + i], o, A);
      sub3(m->X + 3 * m->fvert[b + (i + 1) % I], o, E);
      double T[4][3];
      const double* pts[4] = {r, p0, out ? A : E, out ? E : A};
      for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) T[a][d] = pts[a][d];
      double d6 = det6(T[0], T[1], T[2], T[3]);
      /* two sub3, det6, four planes (two sub3, cross, scale, dot) and the
       * PLIC plane */
      ORC_FLOPS(6 + 23 + 4 * 23 + (tag == 0 ? 9 : 0) + 2);
      if (d6 == 0.0) continue;
      double sg = d6 > 0 ? 1.0 : -1.0;
      /* the 4 inward planes of tetrahedron T */
      int np2 = 0;
      static const int opp[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
      for (int a = 0; a < 4; ++a) {
        double u[3], w[3], nn[3];
        sub3(T[opp[a][1]], T[opp[a][0]], u);
        sub3(T[opp[a][2]], T[opp[a][0]], w);
        cross3(u, w, nn); /* outward for a positive tetrahedron */
        for (int d = 0; d < 3; ++d) nn[d] *= sg;
        planes[4 * np2] = -nn[0]; planes[4 * np2 + 1] = -nn[1]; planes[4 * np2 + 2] = -nn[2];
        planes[4 * np2 + 3] = dot3(nn, T[opp[a][0]]);
        ++np2;
      }
      if (tag == 0) {
        const double* n = nrm + 3 * k;
        double d[3];
        sub3(o, m->cc + 3 * k, d);
        planes[4 * np2] = n[0]; planes[4 * np2 + 1] = n[1]; planes[4 * np2 + 2] = n[2];
        planes[4 * np2 + 3] = dot3(n, d) + Cp[k];
        ++np2;
      }
      vol += sg * orc_poly_clip_volume(nv, V, nf, fp, fi, np2, planes);
    }
  }
  return vol;
}

/* ------------------------------------------------------ faceflux (Sec 3.5) */
void orc_faceflux(const orc_mesh* m, const orc_velocity* vel, double t, double dt,
                  const double* F, const int8_t* tag_f, const int8_t* tag_c,
                  const double* nrm, const double* Cp, double* Vd, double* VF,
                  int64_t* stats, int method) {
  (void)F;
  double th = t + 0.5 * dt;
  int64_t n_geo = 0, n_deg = 0, n_edge = 0, n_trunc = 0, n_flops = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : n_geo, n_deg, n_edge, n_trunc, n_flops)
  for (int64_t f = 0; f < m->nf; ++f) {
    double c[3];
    memcpy(c, m->fc + 3 * f, sizeof c);
    double uc[3];
    orc_velocity_eval(vel, c, th, uc);
    double vd = dot3(uc, m->fn + 3 * f) * m->fa[f] * dt;
    Vd[f] = vd;
    if (tag_f[f] == -1) { VF[f] = 0.0; continue; }
    if (tag_f[f] == 1) { VF[f] = vd; continue; }
    ++n_geo;
    double P[97 * 3];
    double vdd;
    int flags;
    int I = method == 1   ? orc_emfpa(m, f, vel, th, dt, P, 32, &vdd, &flags)
            : method == 2 ? orc_nmfpa(m, f, vel, th, dt, P, 32, &vdd, &flags)
                          : orc_fmfpa(m, f, vel, th, dt, P, 32, &vdd, &flags);
    if (flags & 1) ++n_deg;
    if (flags & 2) ++n_edge;
    int nvp = method == 1 ? 3 * I + 1 : method == 2 ? 2 * I : 2 * I + 1;
    /* local frame at the face centroid */
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < nvp; ++i)
      for (int d = 0; d < 3; ++d) {
        double xv = P[3 * i + d];
        if (xv < lo[d]) lo[d] = xv;
        if (xv > hi[d]) hi[d] = xv;
        P[3 * i + d] = xv - c[d];
      }
    int fp[5 * 32 + 2], fi[16 * 32];
    int nfp = flux_loops(method, I, fp, fi);
    int32_t cand[4096];
    int nc = orc_candidates(m, f, cand, 4096);
    if (nc > 4096) nc = 4096;
    double vf = 0.0;
    for (int q = 0; q < nc; ++q) {
      int32_t kc = cand[q];
      if (tag_c[kc] == -1) continue;
      const double* bb = m->bbox + 6 * kc;
      if (!(hi[0] > bb[0] && lo[0] < bb[3] && hi[1] > bb[1] && lo[1] < bb[4] &&
            hi[2] > bb[2] && lo[2] < bb[5]))
        continue;
      ++n_trunc;
      const int64_t f0 = g_flops;
      vf += truncate_in_cell(m, nvp, P, nfp, fp, fi, kc, tag_c[kc], nrm, Cp, c);
      n_flops += g_flops - f0 + 1;  /* and the sum over cells */
    }
    VF[f] = vf;
  }
  if (stats) {
    stats[0] = n_geo; stats[1] = n_deg; stats[2] = n_edge; stats[3] = n_trunc; stats[4] = n_flops;
  }
}

/* --------------------------------------------------------- vofadv (Eq fnext) */
void orc_vofadv(const orc_mesh* m, const double* Vd, const double* VF, double* F) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < m->nc; ++c) {
    double vdt = 0.0, vft = 0.0;
    for (int64_t q = m->cf_ptr[c]; q < m->cf_ptr[c + 1]; ++q) {
      int32_t f = m->cf[q];
      double s = (m->own[f] == c) ? 1.0 : -1.0;
      vdt += s * Vd[f];
      vft += s * VF[f];
    }
    double V = m->cvol[c];
    double fn = (F[c] * (1.0 + vdt / (2.0 * V)) - vft / V) / (1.0 - vdt / (2.0 * V));
    F[c] = fmax(fmin(fn, 1.0), 0.0);
  }
}

/* ------------------------------------------------------ time step (Eq eq:cfl) */
static void max_face_speed(const orc_mesh* m, const orc_velocity* v, double t, double um[3]) {
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m0, m1, m2)
  for (int64_t f = 0; f < m->nf; ++f) {
    double u[3];
    orc_velocity_eval(v, m->fc + 3 * f, t, u);
    if (fabs(u[0]) > m0) m0 = fabs(u[0]);
    if (fabs(u[1]) > m1) m1 = fabs(u[1]);
    if (fabs(u[2]) > m2) m2 = fabs(u[2]);
  }
  um[0] = m0; um[1] = m1; um[2] = m2;
}

static double dt_from(const double hmin[3], const double um[3], double cfl) {
  double dt = 1e300;
  for (int d = 0; d < 3; ++d)
    if (um[d] > 0.0) {
      double x = hmin[d] / um[d];
      if (x < dt) dt = x;
    }
  return dt * cfl;
}

double orc_suggest_dt(const orc_mesh* m, const orc_velocity* v, double t, double cfl,
                      double t_end) {
  double hmin[3] = {1e300, 1e300, 1e300};
  for (int64_t c = 0; c < m->nc; ++c)
    for (int d = 0; d < 3; ++d) {
      double h = m->bbox[6 * c + 3 + d] - m->bbox[6 * c + d];
      if (h < hmin[d]) hmin[d] = h;
    }
  double um[3];
  max_face_speed(m, v, t, um);
  double dt = dt_from(hmin, um, cfl);
  if (t + dt > t_end) dt = t_end - t;
  double um2[3];
  max_face_speed(m, v, t + dt, um2);
  for (int d = 0; d < 3; ++d)
    if (um2[d] > um[d]) um[d] = um2[d];
  double dt2 = dt_from(hmin, um, cfl);
  if (dt2 < dt) dt = dt2;
  if (t + dt > t_end) dt = t_end - t;
  return dt;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

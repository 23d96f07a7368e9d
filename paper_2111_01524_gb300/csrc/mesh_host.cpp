// Host-side derived connectivity of a face-based mesh (the neigbcell routine
// and the cell/face/node incidence used by compgrid, Sec. 3.1), built once
// per context with O(N) counting passes, parallel over cells (OpenMP).
#include "mesh_host.h"

#include <algorithm>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace gvof {

static void exclusive_scan(std::vector<int64_t>& a) {
  int64_t s = 0;
  for (auto& x : a) {
    int64_t t = x;
    x = s;
    s += t;
  }
}

bool build_connectivity(int64_t nv, int64_t nf, int64_t nc, const int64_t* fptr,
                        const int32_t* fvert, const int32_t* own, const int32_t* nbr,
                        HostConn& out, std::string& err) {
  // cell -> faces (ascending face id; neighbour side stored as ~f)
  out.cf_ptr.assign(nc + 1, 0);
  for (int64_t f = 0; f < nf; ++f) {
    out.cf_ptr[own[f] + 1]++;
    if (nbr[f] >= 0) out.cf_ptr[nbr[f] + 1]++;
  }
  for (int64_t c = 0; c < nc; ++c) out.cf_ptr[c + 1] += out.cf_ptr[c];
  out.cf.resize(out.cf_ptr[nc]);
  {
    std::vector<int64_t> fill(out.cf_ptr.begin(), out.cf_ptr.end() - 1);
    for (int64_t f = 0; f < nf; ++f) {
      out.cf[fill[own[f]]++] = (int32_t)f;
      if (nbr[f] >= 0) out.cf[fill[nbr[f]]++] = ~(int32_t)f;
    }
  }
  for (int64_t c = 0; c < nc; ++c) {
    int64_t n = out.cf_ptr[c + 1] - out.cf_ptr[c];
    if (n < 4) {
      err = "cell " + std::to_string(c) + " has fewer than 4 faces";
      return false;
    }
  }
  // cell -> vertices (sorted unique)
  std::vector<int64_t> cnt(nc + 1, 0);
  out.cv_ptr.assign(nc + 1, 0);
  std::vector<int64_t> raw_ptr(nc + 1, 0);
  for (int64_t c = 0; c < nc; ++c) {
    int64_t s = 0;
    for (int64_t q = out.cf_ptr[c]; q < out.cf_ptr[c + 1]; ++q) {
      int32_t fs = out.cf[q];
      int32_t f = fs >= 0 ? fs : ~fs;
      s += fptr[f + 1] - fptr[f];
    }
    raw_ptr[c + 1] = raw_ptr[c] + s;
  }
  std::vector<int32_t> raw(raw_ptr[nc]);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t p = raw_ptr[c];
    for (int64_t q = out.cf_ptr[c]; q < out.cf_ptr[c + 1]; ++q) {
      int32_t fs = out.cf[q];
      int32_t f = fs >= 0 ? fs : ~fs;
      for (int64_t k = fptr[f]; k < fptr[f + 1]; ++k) raw[p++] = fvert[k];
    }
    std::sort(raw.begin() + raw_ptr[c], raw.begin() + raw_ptr[c + 1]);
    cnt[c] = std::unique(raw.begin() + raw_ptr[c], raw.begin() + raw_ptr[c + 1]) -
             (raw.begin() + raw_ptr[c]);
  }
  for (int64_t c = 0; c < nc; ++c) out.cv_ptr[c + 1] = out.cv_ptr[c] + cnt[c];
  out.cv.resize(out.cv_ptr[nc]);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c)
    std::memcpy(out.cv.data() + out.cv_ptr[c], raw.data() + raw_ptr[c], sizeof(int32_t) * cnt[c]);
  std::vector<int32_t>().swap(raw);
  // vertex -> cells (ascending cell id)
  out.vc_ptr.assign(nv + 1, 0);
  for (int64_t q = 0; q < out.cv_ptr[nc]; ++q) out.vc_ptr[out.cv[q] + 1]++;
  for (int64_t v = 0; v < nv; ++v) out.vc_ptr[v + 1] += out.vc_ptr[v];
  out.vc.resize(out.vc_ptr[nv]);
  {
    std::vector<int64_t> fill(out.vc_ptr.begin(), out.vc_ptr.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int64_t q = out.cv_ptr[c]; q < out.cv_ptr[c + 1]; ++q)
        out.vc[fill[out.cv[q]]++] = (int32_t)c;
  }
  for (int64_t v = 0; v < nv; ++v)
    if (out.vc_ptr[v + 1] == out.vc_ptr[v]) {
      err = "vertex " + std::to_string(v) + " belongs to no cell";
      return false;
    }
  // neigbcell: cells sharing >= 1 node, self excluded, ascending
  std::vector<int64_t> ncnt(nc, 0);
  int nthreads = 1;
#ifdef _OPENMP
  nthreads = omp_get_max_threads();
#endif
  // pass 1: counts
#pragma omp parallel
  {
    std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t c = 0; c < nc; ++c) {
      buf.clear();
      for (int64_t q = out.cv_ptr[c]; q < out.cv_ptr[c + 1]; ++q) {
        int32_t v = out.cv[q];
        buf.insert(buf.end(), out.vc.begin() + out.vc_ptr[v], out.vc.begin() + out.vc_ptr[v + 1]);
      }
      std::sort(buf.begin(), buf.end());
      int64_t u = std::unique(buf.begin(), buf.end()) - buf.begin();
      ncnt[c] = u - 1;
    }
  }
  (void)nthreads;
  out.nb_ptr.assign(nc + 1, 0);
  for (int64_t c = 0; c < nc; ++c) out.nb_ptr[c + 1] = out.nb_ptr[c] + ncnt[c];
  out.nb.resize(out.nb_ptr[nc]);
#pragma omp parallel
  {
    std::vector<int32_t> buf;
#pragma omp for schedule(dynamic, 1024)
    for (int64_t c = 0; c < nc; ++c) {
      buf.clear();
      for (int64_t q = out.cv_ptr[c]; q < out.cv_ptr[c + 1]; ++q) {
        int32_t v = out.cv[q];
        buf.insert(buf.end(), out.vc.begin() + out.vc_ptr[v], out.vc.begin() + out.vc_ptr[v + 1]);
      }
      std::sort(buf.begin(), buf.end());
      auto e = std::unique(buf.begin(), buf.end());
      int64_t p = out.nb_ptr[c];
      for (auto it = buf.begin(); it != e; ++it)
        if (*it != (int32_t)c) out.nb[p++] = *it;
    }
  }
  out.max_cell_faces = 0;
  out.max_cell_verts = 0;
  out.max_cell_entries = 0;
  for (int64_t c = 0; c < nc; ++c) {
    int nfc = (int)(out.cf_ptr[c + 1] - out.cf_ptr[c]);
    int ncv = (int)(out.cv_ptr[c + 1] - out.cv_ptr[c]);
    int ent = (int)(raw_ptr[c + 1] - raw_ptr[c]);
    out.max_cell_faces = std::max(out.max_cell_faces, nfc);
    out.max_cell_verts = std::max(out.max_cell_verts, ncv);
    out.max_cell_entries = std::max(out.max_cell_entries, ent);
  }
  return true;
}

void join_connectivity(const std::vector<const HostConn*>& parts, const std::vector<int64_t>& co,
                       const std::vector<int64_t>& fo, const std::vector<int64_t>& vo, HostConn& out) {
  const int ng = (int)parts.size();
  // one CSR: grid g's rows follow grid g-1's, offsets shifted by the entries
  // before it, entries shifted by shift(g, x)
  auto join = [&](std::vector<int64_t>& ptr, std::vector<int32_t>& idx,
                  const std::vector<int64_t> HostConn::*pp, const std::vector<int32_t> HostConn::*pi,
                  const std::vector<int64_t>& rows, auto shift) {
    int64_t tot = 0;
    for (int g = 0; g < ng; ++g) tot += (parts[g]->*pi).size();
    ptr.assign(rows[ng] + 1, 0);
    idx.resize(tot);
    int64_t e0 = 0;
    for (int g = 0; g < ng; ++g) {
      const std::vector<int64_t>& p = parts[g]->*pp;
      const std::vector<int32_t>& x = parts[g]->*pi;
      const int64_t nr = rows[g + 1] - rows[g];
      for (int64_t r = 0; r <= nr; ++r) ptr[rows[g] + r] = e0 + p[r];
      for (size_t k = 0; k < x.size(); ++k) idx[e0 + k] = shift(g, x[k]);
      e0 += (int64_t)x.size();
    }
  };
  join(out.cf_ptr, out.cf, &HostConn::cf_ptr, &HostConn::cf, co, [&](int g, int32_t f) {
    return f >= 0 ? (int32_t)(f + fo[g]) : ~(int32_t)(~f + fo[g]);
  });
  join(out.cv_ptr, out.cv, &HostConn::cv_ptr, &HostConn::cv, co,
       [&](int g, int32_t v) { return (int32_t)(v + vo[g]); });
  join(out.vc_ptr, out.vc, &HostConn::vc_ptr, &HostConn::vc, vo,
       [&](int g, int32_t c) { return (int32_t)(c + co[g]); });
  join(out.nb_ptr, out.nb, &HostConn::nb_ptr, &HostConn::nb, co,
       [&](int g, int32_t c) { return (int32_t)(c + co[g]); });
  out.max_cell_faces = out.max_cell_verts = out.max_cell_entries = 0;
  for (const HostConn* h : parts) {
    out.max_cell_faces = std::max(out.max_cell_faces, h->max_cell_faces);
    out.max_cell_verts = std::max(out.max_cell_verts, h->max_cell_verts);
    out.max_cell_entries = std::max(out.max_cell_entries, h->max_cell_entries);
  }
}

}  // namespace gvof

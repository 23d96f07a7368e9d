// Serving: continuous batching of "advance this interface N steps" requests
// (vof_server_*), and the exact device footprint of a context
// (vof_estimate_bytes), which the server admits requests against.
//
// Requests are admitted as slots of batched contexts (vof_batch_create): at
// each scheduling tick the queued requests that fit the device budget, in
// arrival order, become the grids of one new context, which keeps their
// meshes and states on the device until all of them are done. Each live
// batch advances one step per tick through its captured CUDA graph on its
// own stream, with every slot's own velocity field, time and time step (a
// slot whose request is done moves no more: its time step is 0), so the
// batches' work overlaps on the device. A request's result (its slice of F)
// is copied back asynchronously after its last step. A grid's arithmetic is
// the same alone and in a batch, so each result equals the request run
// alone, bit for bit.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <vector>

#include "mesh_host.h"
#include "vof_common.cuh"

using namespace gvof;

namespace {

// device bytes of one context (every allocation of vof_batch_create), from
// the mesh sizes and the connectivity counts
struct CtxSizes {
  int64_t nv, nf, nc, nfv, ncf, ncv, nvc, nnb, nbf;
  int ng;
};

template <typename T>
int64_t bytes_of(int64_t n) {
  return (int64_t)sizeof(T) * (n > 0 ? n : 1);
}

int64_t context_bytes(const CtxSizes& z, const vof_options& o) {
  const int64_t nv = z.nv, nf = z.nf, nc = z.nc;
  int64_t b = 0;
  b += 3 * bytes_of<double>(nv);                                       // x y z
  b += bytes_of<int64_t>(nf + 1) + bytes_of<int32_t>(z.nfv);           // face CSR
  b += 2 * bytes_of<int32_t>(nf);                                      // owner, neighbour
  b += 7 * bytes_of<double>(nf);                                       // face geometry
  b += bytes_of<int64_t>(nc + 1) + bytes_of<int32_t>(z.ncf);           // cell -> faces
  b += bytes_of<int64_t>(nc + 1) + bytes_of<int32_t>(z.ncv);           // cell -> vertices
  b += bytes_of<int64_t>(nv + 1) + bytes_of<int32_t>(z.nvc);           // vertex -> cells
  b += bytes_of<int64_t>(nc + 1) + bytes_of<int32_t>(z.nnb);           // neigbcell
  b += 4 * bytes_of<double>(nc) + bytes_of<double>(6 * nc) + bytes_of<uint8_t>(nc);  // cell geometry
  b += bytes_of<double>(nc) + 4 * bytes_of<double>(nc);                // F, planes
  b += bytes_of<int8_t>(nv) + bytes_of<int8_t>(nf) + bytes_of<int8_t>(nc);  // tags
  b += 3 * bytes_of<double>(nf);                                       // V_d, V_F, rate
  b += bytes_of<int32_t>(nc) + bytes_of<int32_t>(nf);                  // lists
  b += bytes_of<unsigned long long>(kNCnt) + bytes_of<double>(kRedSlots) +
       bytes_of<double>(kNAcc * kAccSlots);
  b += bytes_of<int64_t>(nv + 1) + bytes_of<int32_t>(z.nfv);           // node -> faces
  b += bytes_of<int32_t>(nc) + bytes_of<int32_t>(nv) + bytes_of<int32_t>(nf);  // stamps
  b += bytes_of<int32_t>(nc) + bytes_of<int32_t>(nv);                  // band lists
  b += bytes_of<int32_t>(z.nbf > 0 ? z.nbf : 1);                       // boundary faces
  const int64_t rep_cap = std::min<int64_t>(nf, kFmCap);
  if (o.precision == VOF_PREC_MIXED) {
    b += 3 * bytes_of<float2>(nv) + 3 * bytes_of<float2>(nf) + 3 * bytes_of<float>(nf) +
         bytes_of<float>(nf);
    b += 3 * bytes_of<float2>(nc) + bytes_of<float2>(6 * nc) + bytes_of<float>(nc);
    b += 4 * bytes_of<float>(nc) + bytes_of<float4>(z.ncf);
    b += bytes_of<uint8_t>(nf) + bytes_of<double>(nc) + bytes_of<int32_t>(nc);
    b += 2 * bytes_of<double>(nc);
    b += bytes_of<int32_t>(rep_cap) + bytes_of<int32_t>(2 * rep_cap) + bytes_of<int32_t>(nc);
  }
  b += bytes_of<double>(6 * z.ng);                                     // domain boxes
  const int64_t fm_cap = o.poly_capacity > 0 ? std::min<int64_t>(nf, o.poly_capacity)
                                             : std::min<int64_t>(nf, kFmCap);
  const int64_t gs = o.precision == VOF_PREC_MIXED ? 4 : 8;
  b += gs * (3 * kFmSlots + 7) * fm_cap;                               // prebuilt polyhedra
  b += 2 * bytes_of<uint32_t>(fm_cap) + bytes_of<uint8_t>(nf);         // meta, split, coverage
  if (cand_lists_on(o, z.nnb, nc))
    b += bytes_of<int32_t>(kPreCand * fm_cap) + bytes_of<uint8_t>(fm_cap);  // candidate lists
  if (o.reconstruction == VOF_RECON_LSFIR) {
    b += o.precision == VOF_PREC_MIXED ? 6 * bytes_of<float>(nc) : 6 * bytes_of<double>(nc);
    b += bytes_of<unsigned long long>(kMaxLsfirIter + 1);
  }
  b += bytes_of<float>(nv);                                            // star radii
  b += bytes_of<int64_t>(z.ng + 1) + bytes_of<GridParam>(z.ng) +
       bytes_of<unsigned long long>(3 * z.ng);
  return b;
}

thread_local std::string s_err;

vof_status sfail(vof_status s, const std::string& m) {
  s_err = m;
  gvof::set_last_error(m.c_str());
  return s;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct MeshCopy {
  int64_t nv = 0, nf = 0, nc = 0;
  std::vector<double> X;
  std::vector<int64_t> fp;
  std::vector<int32_t> fv, own, nbr;
  vof_mesh_desc desc() const {
    vof_mesh_desc d;
    d.n_vert = nv; d.n_face = nf; d.n_cell = nc;
    d.X = X.data(); d.face_ptr = fp.data(); d.face_vert = fv.data();
    d.owner = own.data(); d.neighbour = nbr.data();
    return d;
  }
};

enum { kQueued = 0, kRunning = 1, kDone = 2 };

struct Request {
  int64_t id;
  MeshCopy mesh;
  std::vector<double> F0;
  vof_velocity vel;
  int n_steps;
  double cfl, t_end;
  int64_t bytes = -1;               // device footprint alone (sized at admission)
  std::unique_ptr<HostConn> conn;   // its connectivity, built once, until its batch exists
  std::string refused;              // why admission refused it (empty: not refused)
  int state = kQueued;
  int batch = -1, slot = -1;
  int k = 0;            // steps queued
  double t = 0.0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  double* pinned = nullptr;  // result copy
  cudaEvent_t done_ev = nullptr;
  bool copy_queued = false;
  std::vector<double> result;
};

struct Batch {
  vof_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<int64_t> reqs;  // request index per slot
  std::vector<int64_t> cell_off;
  int64_t bytes = 0;
  bool live = true;
};

}  // namespace

struct vof_server {
  vof_server_options opt;
  vof_options copt;
  int64_t budget = 0;
  std::vector<Request> reqs;
  std::deque<int64_t> queue;
  std::vector<Batch> batches;
  int64_t bytes_live = 0, peak_bytes = 0, max_active = 0, n_batches = 0, batch_steps = 0;
  int64_t cell_steps = 0;
  double t0 = -1.0;
};

extern "C" {

vof_status vof_estimate_bytes(const vof_mesh_desc* meshes, int n_grids, const vof_options* opt,
                              int64_t* bytes) {
  if (!meshes || n_grids < 1 || !bytes) return sfail(VOF_EINVAL, "bad arguments");
  vof_options o;
  if (opt) o = *opt;
  else { std::memset(&o, 0, sizeof o); o.precision = VOF_PREC_FP64; }
  CtxSizes z{};
  z.ng = n_grids;
  for (int g = 0; g < n_grids; ++g) {
    const vof_mesh_desc& m = meshes[g];
    if (!m.X || !m.face_ptr || !m.face_vert || !m.owner || !m.neighbour || m.n_vert <= 0 ||
        m.n_face <= 0 || m.n_cell <= 0)
      return sfail(VOF_EINVAL, "grid " + std::to_string(g) + ": empty or NULL mesh");
    HostConn hc;
    std::string err;
    if (!build_connectivity(m.n_vert, m.n_face, m.n_cell, m.face_ptr, m.face_vert, m.owner,
                            m.neighbour, hc, err))
      return sfail(VOF_EINVAL, err);
    z.nv += m.n_vert; z.nf += m.n_face; z.nc += m.n_cell; z.nfv += m.face_ptr[m.n_face];
    z.ncf += hc.cf_ptr[m.n_cell]; z.ncv += hc.cv_ptr[m.n_cell]; z.nvc += hc.vc_ptr[m.n_vert];
    z.nnb += hc.nb_ptr[m.n_cell];
    for (int64_t f = 0; f < m.n_face; ++f) z.nbf += m.neighbour[f] < 0;
  }
  *bytes = context_bytes(z, o);
  return VOF_OK;
}

vof_status vof_server_create(const vof_server_options* opt, vof_server** out) {
  if (!opt || !out) return sfail(VOF_EINVAL, "NULL argument");
  *out = nullptr;
  if (opt->precision != VOF_PREC_FP64 && opt->precision != VOF_PREC_MIXED)
    return sfail(VOF_EINVAL, "bad precision");
  if (opt->budget_bytes < 0 || opt->max_batch < 0) return sfail(VOF_EINVAL, "bad budget or batch size");
  if (opt->reserved[0] != 0 || opt->reserved[1] != 0)
    return sfail(VOF_EINVAL, "reserved options must be zero");
  vof_server* s = new vof_server();
  s->opt = *opt;
  std::memset(&s->copt, 0, sizeof s->copt);
  s->copt.eps = 1e-12;
  s->copt.beta = 1.5;
  s->copt.precision = opt->precision;
  s->copt.flux_polyhedron = opt->flux_polyhedron;
  s->copt.reconstruction = opt->reconstruction;
  s->budget = opt->budget_bytes;
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return sfail(VOF_ECUDA, "cudaMemGetInfo failed");
    }
    s->budget = (int64_t)(0.8 * (double)fr);
  }
  *out = s;
  return VOF_OK;
}

vof_status vof_server_submit(vof_server* s, const vof_mesh_desc* mesh, const double* F0,
                             const vof_velocity* vel, int32_t n_steps, double cfl, double t_end,
                             int64_t* id) {
  if (!s || !mesh || !F0 || !vel || !id) return sfail(VOF_EINVAL, "NULL argument");
  if (n_steps < 1 || !(cfl > 0.0) || !(t_end > 0.0)) return sfail(VOF_EINVAL, "bad steps, cfl or t_end");
  if (vel->kind < VOF_VEL_DEFORMATION || vel->kind > VOF_VEL_DEFORMATION2D)
    return sfail(VOF_EINVAL, "unknown velocity kind");
  Request r;
  r.id = (int64_t)s->reqs.size();
  MeshCopy& m = r.mesh;
  m.nv = mesh->n_vert; m.nf = mesh->n_face; m.nc = mesh->n_cell;
  if (m.nv <= 0 || m.nf <= 0 || m.nc <= 0 || !mesh->X || !mesh->face_ptr || !mesh->face_vert ||
      !mesh->owner || !mesh->neighbour)
    return sfail(VOF_EINVAL, "empty or NULL mesh");
  m.X.assign(mesh->X, mesh->X + 3 * m.nv);
  m.fp.assign(mesh->face_ptr, mesh->face_ptr + m.nf + 1);
  m.fv.assign(mesh->face_vert, mesh->face_vert + m.fp[m.nf]);
  m.own.assign(mesh->owner, mesh->owner + m.nf);
  m.nbr.assign(mesh->neighbour, mesh->neighbour + m.nf);
  r.F0.assign(F0, F0 + m.nc);
  r.vel = *vel;
  r.n_steps = n_steps;
  r.cfl = cfl;
  r.t_end = t_end;
  // structure checks here; the connectivity (and with it the footprint) is
  // built once, when the request reaches the front of the queue
  if (m.fp[0] != 0) return sfail(VOF_EINVAL, "face_ptr[0] != 0");
  for (int64_t f = 0; f < m.nf; ++f) {
    if (m.fp[f + 1] < m.fp[f] + 3) return sfail(VOF_EINVAL, "a face has fewer than 3 nodes");
    if (m.own[f] < 0 || m.own[f] >= m.nc || m.nbr[f] < -1 || m.nbr[f] >= m.nc || m.nbr[f] == m.own[f])
      return sfail(VOF_EINVAL, "bad owner/neighbour");
  }
  for (int32_t v : m.fv)
    if (v < 0 || v >= m.nv) return sfail(VOF_EINVAL, "face_vert entry out of range");
  r.t_submit = now_s();
  if (s->t0 < 0) s->t0 = r.t_submit;
  *id = r.id;
  s->reqs.push_back(std::move(r));
  s->queue.push_back(*id);
  return VOF_OK;
}

#define SCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return sfail(VOF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static vof_status retire(vof_server* s) {
  // results whose copies completed; batches with every request done
  for (Request& r : s->reqs) {
    if (r.state != kRunning || !r.copy_queued) continue;
    cudaError_t q = cudaEventQuery(r.done_ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return sfail(VOF_ECUDA, cudaGetErrorString(q));
    r.result.assign(r.pinned, r.pinned + r.mesh.nc);
    cudaFreeHost(r.pinned);
    r.pinned = nullptr;
    cudaEventDestroy(r.done_ev);
    r.done_ev = nullptr;
    r.state = kDone;
    r.t_done = now_s();
    s->cell_steps += r.mesh.nc * (int64_t)r.n_steps;
  }
  for (Batch& b : s->batches) {
    if (!b.live) continue;
    bool all = true;
    for (int64_t q : b.reqs) all &= s->reqs[q].state == kDone;
    if (!all) continue;
    SCK(cudaStreamSynchronize(b.stream));
    vof_destroy(b.ctx);
    cudaStreamDestroy(b.stream);
    b.ctx = nullptr;
    b.stream = nullptr;
    b.live = false;
    s->bytes_live -= b.bytes;
  }
  return VOF_OK;
}

// the connectivity and the device footprint of request r alone
static vof_status size_request(vof_server* s, Request& r) {
  if (r.bytes >= 0) return VOF_OK;
  r.conn.reset(new HostConn());
  std::string err;
  const MeshCopy& m = r.mesh;
  if (!build_connectivity(m.nv, m.nf, m.nc, m.fp.data(), m.fv.data(), m.own.data(), m.nbr.data(),
                          *r.conn, err)) {
    r.conn.reset();
    r.refused = err;
    return sfail(VOF_EINVAL, "request " + std::to_string(r.id) + ": " + err);
  }
  CtxSizes z{};
  z.ng = 1;
  z.nv = m.nv; z.nf = m.nf; z.nc = m.nc; z.nfv = m.fp[m.nf];
  z.ncf = r.conn->cf_ptr[m.nc]; z.ncv = r.conn->cv_ptr[m.nc]; z.nvc = r.conn->vc_ptr[m.nv];
  z.nnb = r.conn->nb_ptr[m.nc];
  for (int64_t f = 0; f < m.nf; ++f) z.nbf += m.nbr[f] < 0;
  r.bytes = context_bytes(z, s->copt);
  return VOF_OK;
}

static vof_status admit(vof_server* s) {
  std::vector<int64_t> take;
  int64_t need = 0;
  while (!s->queue.empty()) {
    Request& r = s->reqs[s->queue.front()];
    if (s->opt.max_batch > 0 && (int)take.size() >= s->opt.max_batch) break;
    if (r.bytes < 0) {
      const vof_status st = size_request(s, r);
      if (st != VOF_OK) {
        s->queue.pop_front();  // refused: poll reports why
        return st;
      }
    }
    // the batch's footprint is at most the sum of its grids' own (the
    // per-context tables are shared), so the sum is admitted against
    if (s->bytes_live + need + r.bytes > s->budget) {
      if (s->bytes_live == 0 && take.empty())
        return sfail(VOF_ENOMEM, "request " + std::to_string(r.id) + " needs " +
                                     std::to_string(r.bytes) + " bytes, above the budget");
      break;
    }
    need += r.bytes;
    take.push_back(s->queue.front());
    s->queue.pop_front();
  }
  if (take.empty()) return VOF_OK;
  Batch b;
  SCK(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
  std::vector<vof_mesh_desc> descs;
  std::vector<const HostConn*> conns;
  std::vector<double> F;
  for (int64_t q : take) {
    descs.push_back(s->reqs[q].mesh.desc());
    conns.push_back(s->reqs[q].conn.get());
    F.insert(F.end(), s->reqs[q].F0.begin(), s->reqs[q].F0.end());
  }
  vof_status st = batch_create_with_conn(descs.data(), (int)descs.size(), &s->copt, b.stream, &b.ctx,
                                         conns.data());
  for (int64_t q : take) s->reqs[q].conn.reset();
  if (st != VOF_OK) { cudaStreamDestroy(b.stream); return st; }
  b.cell_off.resize(take.size() + 1);
  int ng = 0;
  vof_batch_offsets(b.ctx, &ng, b.cell_off.data(), nullptr, nullptr);
  st = vof_set_fraction(b.ctx, F.data(), VOF_MEM_HOST, b.stream);
  if (st == VOF_OK) st = vof_reconstruct(b.ctx, b.stream);
  if (st == VOF_OK) st = vof_graph_capture(b.ctx, 1, b.stream);
  if (st != VOF_OK) { vof_destroy(b.ctx); cudaStreamDestroy(b.stream); return st; }
  b.bytes = vof_device_bytes(b.ctx);
  b.reqs = take;
  const double t = now_s();
  for (size_t i = 0; i < take.size(); ++i) {
    Request& r = s->reqs[take[i]];
    r.state = kRunning;
    r.batch = (int)s->batches.size();
    r.slot = (int)i;
    r.t_admit = t;
  }
  s->bytes_live += b.bytes;
  s->peak_bytes = std::max(s->peak_bytes, s->bytes_live);
  s->batches.push_back(b);
  ++s->n_batches;
  return VOF_OK;
}

static vof_status advance(vof_server* s, int32_t* n_active) {
  int64_t active = 0;
  for (Batch& b : s->batches) {
    if (!b.live) continue;
    const int n = (int)b.reqs.size();
    std::vector<vof_velocity> vels(n);
    std::vector<double> t(n), dt(n, 0.0), tend(n), one(n);
    std::vector<char> moving(n, 0);
    for (int i = 0; i < n; ++i) {
      const Request& r = s->reqs[b.reqs[i]];
      vels[i] = r.vel;
      t[i] = r.t;
      tend[i] = r.t_end;
      moving[i] = r.k < r.n_steps && r.t < r.t_end;
    }
    // Eq. eq:cfl per slot with the slot's own CFL number (one pass per
    // distinct CFL among the batch's slots); a slot whose request is done
    // takes dt = 0 and does not move
    for (int i = 0; i < n; ++i) {
      if (!moving[i] || dt[i] != 0.0) continue;
      const double cfl = s->reqs[b.reqs[i]].cfl;
      vof_status st = vof_suggest_dt_batch(b.ctx, vels.data(), t.data(), cfl, tend.data(), one.data());
      if (st != VOF_OK) return st;
      for (int j = i; j < n; ++j)
        if (moving[j] && s->reqs[b.reqs[j]].cfl == cfl) dt[j] = one[j];
    }
    bool any = false;
    for (int i = 0; i < n; ++i) any |= moving[i] != 0;
    if (!any) continue;
    vof_status st = vof_graph_launch(b.ctx, vels.data(), t.data(), dt.data(), b.stream);
    if (st != VOF_OK) return st;
    ++s->batch_steps;
    for (int i = 0; i < n; ++i) {
      if (!moving[i]) continue;
      Request& r = s->reqs[b.reqs[i]];
      r.t += dt[i];
      ++r.k;
      ++active;
      if (r.k == r.n_steps || !(r.t < r.t_end)) {
        // the request's last step is queued: copy its slice of F back
        const int64_t c0 = b.cell_off[i], nc = b.cell_off[i + 1] - c0;
        SCK(cudaMallocHost((void**)&r.pinned, sizeof(double) * (size_t)nc));
        SCK(cudaEventCreateWithFlags(&r.done_ev, cudaEventDisableTiming));
        SCK(cudaMemcpyAsync(r.pinned, b.ctx->F + c0, sizeof(double) * (size_t)nc,
                            cudaMemcpyDeviceToHost, b.stream));
        SCK(cudaEventRecord(r.done_ev, b.stream));
        r.copy_queued = true;
        r.n_steps = r.k;
      }
    }
  }
  s->max_active = std::max(s->max_active, active);
  if (n_active) *n_active = (int)active;
  return VOF_OK;
}

vof_status vof_server_step(vof_server* s, int32_t* n_active) {
  if (!s) return sfail(VOF_EINVAL, "NULL server");
  vof_status st = retire(s);
  if (st != VOF_OK) return st;
  st = admit(s);
  if (st != VOF_OK) return st;
  return advance(s, n_active);
}

vof_status vof_server_drain(vof_server* s) {
  if (!s) return sfail(VOF_EINVAL, "NULL server");
  for (;;) {
    int32_t act = 0;
    vof_status st = vof_server_step(s, &act);
    if (st != VOF_OK) return st;
    bool pending = !s->queue.empty();
    for (const Request& r : s->reqs) pending |= r.state != kDone;
    if (!pending) return VOF_OK;
    if (act == 0) {
      // only copies in flight: wait for them
      for (Batch& b : s->batches)
        if (b.live) SCK(cudaStreamSynchronize(b.stream));
    }
  }
}

vof_status vof_server_poll(vof_server* s, int64_t id, int32_t* state, double* F,
                           double* latency_s) {
  if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return sfail(VOF_EINVAL, "unknown request");
  vof_status st = retire(s);
  if (st != VOF_OK) return st;
  const Request& r = s->reqs[id];
  if (!r.refused.empty()) return sfail(VOF_EINVAL, "request " + std::to_string(id) + " refused: " + r.refused);
  if (state) *state = r.state;
  if (r.state == kDone) {
    if (F) std::memcpy(F, r.result.data(), sizeof(double) * r.result.size());
    if (latency_s) *latency_s = r.t_done - r.t_submit;
  } else if (latency_s) {
    *latency_s = -1.0;
  }
  return VOF_OK;
}

vof_status vof_server_get_stats(vof_server* s, vof_server_stats* out) {
  if (!s || !out) return sfail(VOF_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof *out);
  std::vector<double> lat;
  double last = s->t0;
  for (const Request& r : s->reqs) {
    out->n_submitted++;
    if (r.state == kQueued) out->n_queued++;
    else if (r.state == kRunning) out->n_active++;
    else {
      out->n_done++;
      lat.push_back(r.t_done - r.t_submit);
      last = std::max(last, r.t_done);
    }
  }
  out->cell_steps = s->cell_steps;
  out->device_bytes = s->bytes_live;
  out->peak_device_bytes = s->peak_bytes;
  out->budget_bytes = s->budget;
  out->n_batches = s->n_batches;
  out->batch_steps = s->batch_steps;
  out->max_active = s->max_active;
  out->elapsed_s = s->t0 >= 0 ? last - s->t0 : 0.0;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      const double x = p * (double)(lat.size() - 1);
      const size_t i = (size_t)x;
      const double f = x - (double)i;
      return i + 1 < lat.size() ? lat[i] * (1.0 - f) + lat[i + 1] * f : lat[i];
    };
    out->p50_latency_s = pct(0.5);
    out->p99_latency_s = pct(0.99);
  }
  return VOF_OK;
}

void vof_server_destroy(vof_server* s) {
  if (!s) return;
  for (Batch& b : s->batches) {
    if (!b.live) continue;
    cudaStreamSynchronize(b.stream);
    vof_destroy(b.ctx);
    cudaStreamDestroy(b.stream);
  }
  for (Request& r : s->reqs) {
    if (r.pinned) cudaFreeHost(r.pinned);
    if (r.done_ev) cudaEventDestroy(r.done_ev);
  }
  delete s;
}

}  // extern "C"

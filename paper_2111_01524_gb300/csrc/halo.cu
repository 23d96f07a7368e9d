// Cell lists of a context for a partitioned grid (domain decomposition): the
// halo cells a part receives, the cells it sends to each neighbouring part
// and the cells it owns. F is gathered over a list into a plain device
// buffer and scattered back from one, so the exchange itself is a copy
// between two contexts on one device or a send/receive between ranks, with
// no peer-memory operand in any kernel. A scattered value enters F as
// vof_set_fraction's values do: the next sweeps stay band-limited only if
// every changed cell was in the band of the last advect.
#include <string>
#include <vector>

#include "vof_common.cuh"

using namespace gvof;

namespace {

constexpr int kListBlocks = kSMs * 2;
constexpr int kListThreads = 256;

vof_status fail(vof_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(VOF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__device__ __forceinline__ uint64_t bits_of(double x) { return (uint64_t)__double_as_longlong(x); }

__global__ void k_list_gather(const double* F, const int32_t* cells, int64_t n, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = F[cells[i]];
}

// F[cells[i]] = in[i]; a changed cell outside the band of the last advect
// makes the next sweeps full ones
__global__ void k_list_scatter(const double* in, const int32_t* cells, int64_t n, double* F,
                               const int32_t* stamp_c, unsigned long long* cnt) {
  const bool band = cnt[kBandCellsOk] != 0;
  const int32_t epoch = (int32_t)cnt[kEpoch];
  int outside = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cells[i];
    const double f = in[i];
    if (bits_of(f) != bits_of(F[c])) {
      F[c] = f;
      outside |= (!band || stamp_c[c] != epoch) ? 1 : 0;
    }
  }
  if (__syncthreads_or(outside) && threadIdx.x == 0) {
    cnt[kBandCellsOk] = 0;
    cnt[kBandNodesOk] = 0;
  }
}

// sum of V_k F_k over a list: a partial per block in a fixed order, then
// the partials in block order (the result does not depend on scheduling)
__global__ void k_list_volume_partial(const double* cvol, const double* F, const int32_t* cells,
                                      int64_t n, double* part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cells[i];
    acc += cvol[c] * F[c];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(GVOF_FULL, acc, o);
  __shared__ double s[kListThreads / 32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kListThreads / 32; ++i) t += s[i];
    part[blockIdx.x] = t;
  }
}

__global__ void k_list_volume_final(double* part, int nb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nb; ++i) t += part[i];
  part[nb] = t;
}

int grid_for_list(int64_t n) {
  const int64_t b = (n + kListThreads - 1) / kListThreads;
  return (int)(b < 1 ? 1 : (b > kListBlocks ? kListBlocks : b));
}

vof_status list_range(const vof_ctx* c, int list, int64_t* a, int64_t* n) {
  if (!c) return fail(VOF_EINVAL, "NULL context");
  if (!c->list_ptr) return fail(VOF_ESTATE, "no cell lists: call vof_halo_lists first");
  const std::vector<int64_t>& p = *c->list_ptr;
  if (list < 0 || list + 1 >= (int)p.size())
    return fail(VOF_EINVAL, "list " + std::to_string(list) + " out of range");
  *a = p[list];
  *n = p[list + 1] - p[list];
  return VOF_OK;
}

}  // namespace

extern "C" {

vof_status vof_halo_lists(vof_ctx* c, int n_lists, const int64_t* ptr, const int32_t* cells) {
  if (!c || n_lists < 0 || (n_lists > 0 && !ptr)) return fail(VOF_EINVAL, "bad arguments");
  if (n_lists > 0 && ptr[0] != 0) return fail(VOF_EINVAL, "ptr[0] must be 0");
  for (int k = 0; k < n_lists; ++k)
    if (ptr[k + 1] < ptr[k]) return fail(VOF_EINVAL, "ptr must be non-decreasing");
  const int64_t total = n_lists > 0 ? ptr[n_lists] : 0;
  if (total > 0 && !cells) return fail(VOF_EINVAL, "cells is NULL");
  for (int64_t i = 0; i < total; ++i)
    if (cells[i] < 0 || cells[i] >= c->nc)
      return fail(VOF_EINVAL, "list entry " + std::to_string(i) + " is not a cell of this context");
  CK(cudaDeviceSynchronize());  // the old lists may still be read by queued work
  if (c->lists) { cudaFree(c->lists); c->bytes -= (int64_t)sizeof(int32_t) * c->n_list_cells; }
  c->lists = nullptr;
  c->n_list_cells = 0;
  if (!c->list_part) {
    CK(cudaMalloc(&c->list_part, sizeof(double) * (kListBlocks + 1)));
    c->bytes += (int64_t)sizeof(double) * (kListBlocks + 1);
  }
  if (total > 0) {
    CK(cudaMalloc(&c->lists, sizeof(int32_t) * total));
    c->bytes += (int64_t)sizeof(int32_t) * total;
    CK(cudaMemcpy(c->lists, cells, sizeof(int32_t) * total, cudaMemcpyHostToDevice));
  }
  c->n_list_cells = total;
  if (!c->list_ptr) c->list_ptr = new std::vector<int64_t>();
  if (n_lists > 0) c->list_ptr->assign(ptr, ptr + n_lists + 1);
  else c->list_ptr->assign(1, 0);
  return VOF_OK;
}

vof_status vof_halo_export(vof_ctx* c, int list, double* out, void* stream) {
  int64_t a = 0, n = 0;
  vof_status st = list_range(c, list, &a, &n);
  if (st != VOF_OK) return st;
  if (n == 0) return VOF_OK;
  if (!out) return fail(VOF_EINVAL, "out is NULL");
  k_list_gather<<<grid_for_list(n), kListThreads, 0, (cudaStream_t)stream>>>(c->F, c->lists + a,
                                                                             n, out);
  CK(cudaGetLastError());
  return VOF_OK;
}

vof_status vof_halo_import(vof_ctx* c, int list, const double* in, void* stream) {
  int64_t a = 0, n = 0;
  vof_status st = list_range(c, list, &a, &n);
  if (st != VOF_OK) return st;
  if (n == 0) return VOF_OK;
  if (!in) return fail(VOF_EINVAL, "in is NULL");
  k_list_scatter<<<grid_for_list(n), kListThreads, 0, (cudaStream_t)stream>>>(
      in, c->lists + a, n, c->F, c->stamp_c, c->cnt);
  CK(cudaGetLastError());
  c->recon_valid = false;
  return VOF_OK;
}

vof_status vof_list_volume(vof_ctx* c, int list, double* vol, void* stream) {
  int64_t a = 0, n = 0;
  vof_status st = list_range(c, list, &a, &n);
  if (st != VOF_OK) return st;
  if (!vol) return fail(VOF_EINVAL, "vol is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = grid_for_list(n);
  k_list_volume_partial<<<nb, kListThreads, 0, s>>>(c->cvol, c->F, c->lists + a, n, c->list_part);
  k_list_volume_final<<<1, 32, 0, s>>>(c->list_part, nb);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(c->pinned, c->list_part + nb, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *vol = *(const double*)c->pinned;
  return VOF_OK;
}

}  // extern "C"

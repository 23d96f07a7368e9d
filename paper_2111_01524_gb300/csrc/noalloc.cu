// Allocation-free variant of the fixed-order weighted sum sum_i w_i F_i
// (the global fluid volume sum_i V_i F_i when w holds the cell volumes).
//
// Some callers cannot allocate device memory at the point where they need
// this sum: a solver that reserved its whole device budget up front and
// hands out only what it owns, code that must not pay the device-wide
// synchronisation or the failure modes of cudaMalloc in the middle of a
// time step, or a host thread that drives the GPU under a memory policy
// that forbids new allocations. This entry point serves them: the caller
// passes its own input and output device buffers, and the only scratch is
// the file-scope device array below, which every GPU that loads the library
// holds until the process exits.
#include <mutex>
#include <string>

#include "vof_common.cuh"

namespace gvof {
namespace {

constexpr int kChunk = 4096;                  // elements per partial sum
constexpr int kMaxChunks = 65536;             // partial sums held by the scratch
constexpr int64_t kMaxN = (int64_t)kChunk * kMaxChunks;  // 268,435,456 elements
constexpr int kMaxDevices = 64;

// per-chunk partial sums; 512 KiB on every device that loads the library
static __device__ __align__(256) double g_noalloc_scratch[kMaxChunks];

// one block per chunk: each thread sums a fixed strided subset, then a
// fixed-shape tree; the partial of chunk b goes to part[b]
__global__ void k_partial_sums(const double* __restrict__ w, const double* __restrict__ F,
                               int64_t n, double* part) {
  __shared__ double s[256];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  double acc = 0.0;
  for (int i = threadIdx.x; i < kChunk; i += blockDim.x) {
    const int64_t e = base + i;
    if (e < n) acc += w[e] * F[e];
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// one block sums the partials in a fixed order
__global__ void k_final_sum(const double* part, int m, double* out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc += part[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = s[0];
}

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code)
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace gvof

extern "C" vof_status vof_volume_sum_noalloc(const double* w, const double* F, int64_t n,
                                             double* out, void* stream) {
  using namespace gvof;
  if (!w || !F || !out) {
    set_last_error("vof_volume_sum_noalloc: NULL pointer");
    return VOF_EINVAL;
  }
  if (n < 0 || n > kMaxN) {
    set_last_error(("vof_volume_sum_noalloc: n = " + std::to_string(n) + " is outside [0, " +
                    std::to_string(kMaxN) +
                    "] (the fixed scratch holds 65536 partial sums of 4096 elements)").c_str());
    return VOF_EINVAL;
  }
  double* part = nullptr;
  cudaError_t e = scratch_for_current_device(&part);
  if (e != cudaSuccess) {
    set_last_error((std::string("vof_volume_sum_noalloc: scratch set-up: ") +
                    cudaGetErrorString(e)).c_str());
    return VOF_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int m = (int)((n + kChunk - 1) / kChunk);
  if (m > 0) k_partial_sums<<<m, 256, 0, s>>>(w, F, n, part);
  // every partial the final pass reads is written by this call, so nothing
  // left in the scratch by an earlier call is used
  k_final_sum<<<1, 256, 0, s>>>(part, m, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error((std::string("vof_volume_sum_noalloc: launch: ") + cudaGetErrorString(e)).c_str());
    return VOF_ECUDA;
  }
  return VOF_OK;
}

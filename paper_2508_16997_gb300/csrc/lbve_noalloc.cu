// lbve_noalloc.cu -- lbve_field_totals_noalloc: the float64 totals of a
// macroscopic field array, computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host framework whose own allocator
// owns all device memory and forbids side allocations, a latency-critical
// loop that cannot afford the device synchronisation cudaMalloc/cudaFree
// imply, or a caller that only holds a field array and no lbve workspace.
// This entry point serves them: its only scratch (one partial record per
// chunk of nodes) is a file-scope static device array that every GPU loading
// the library keeps until the process exits.  The caller passes the input
// fields and the output buffer.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/lbve.h"
#include "lbve_internal.h"

namespace {

constexpr int kChunk = 1024;       // nodes per partial record
constexpr int kThreadsNA = 256;    // threads per block (4 nodes per thread)
constexpr int kMaxChunks = 16384;  // partial records in the static scratch
constexpr int kSums = 6;           // sum rho, rho ux, rho uy, Axx, Axy, Ayy
constexpr int kRecord = 8;         // doubles per record (6 used, padded)

// Static scratch: 16384 records x 8 doubles = 1 MiB per device.  Shared by
// every call on the device; each call overwrites the records it uses before
// reading them, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxChunks * kRecord];

__device__ __forceinline__ double block_sum(double v, double* s) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreadsNA / 32; ++w) t += s[w];
  return t;  // valid in thread 0
}

// Pass 1: one block per chunk of kChunk nodes writes one partial record.
__global__ void __launch_bounds__(kThreadsNA) chunk_sums(const double* __restrict__ f, int n,
                                                         double* __restrict__ partials) {
  __shared__ double s[kThreadsNA / 32];
  const int base = blockIdx.x * kChunk;
  double v[kSums] = {0, 0, 0, 0, 0, 0};
  for (int j = threadIdx.x; j < kChunk; j += kThreadsNA) {
    const int k = base + j;
    if (k < n) {
      const double rho = f[k];
      v[0] += rho;
      v[1] += rho * f[(size_t)n + k];
      v[2] += rho * f[2 * (size_t)n + k];
      v[3] += f[3 * (size_t)n + k];
      v[4] += f[4 * (size_t)n + k];
      v[5] += f[5 * (size_t)n + k];
    }
  }
  for (int q = 0; q < kSums; ++q) {
    const double t = block_sum(v[q], s);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kRecord + q] = t;
  }
}

// Pass 2: one block sums the records in a fixed order.
__global__ void __launch_bounds__(kThreadsNA) final_sums(const double* __restrict__ partials,
                                                         int n_chunks, double* __restrict__ out) {
  __shared__ double s[kThreadsNA / 32];
  for (int q = 0; q < kSums; ++q) {
    double v = 0.0;
    for (int c = threadIdx.x; c < n_chunks; c += kThreadsNA) v += partials[(size_t)c * kRecord + q];
    const double t = block_sum(v, s);
    if (threadIdx.x == 0) out[q] = t;
  }
}

// Device address of g_partials for each device, looked up once per device
// with that device current (in host code the symbol itself is only a
// host-side stand-in, not a device address).  The cache lives for the
// process: after cudaDeviceReset the module is loaded again and the array
// may move, so the entry point must not be used after a reset.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

}  // namespace

extern "C" int lbve_field_totals_noalloc(const double* d_fields, int32_t nx, int32_t ny,
                                         double* d_out, void* cuda_stream) {
  using lbve::set_error;
  if (!d_fields || !d_out)
    return set_error(LBVE_ERR_ARG, "lbve_field_totals_noalloc: null field or output pointer");
  if (nx < 1 || ny < 1)
    return set_error(LBVE_ERR_ARG, "lbve_field_totals_noalloc: nx = %d, ny = %d must be >= 1",
                     (int)nx, (int)ny);
  const long long n = (long long)nx * ny;
  if (n > (long long)kMaxChunks * kChunk)
    return set_error(LBVE_ERR_ARG,
                     "lbve_field_totals_noalloc: %lld nodes exceed the static scratch limit of "
                     "%d nodes (%d chunks of %d)",
                     n, kMaxChunks * kChunk, kMaxChunks, kChunk);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return set_error(LBVE_ERR_CUDA, "lbve_field_totals_noalloc: cudaGetDevice: %s",
                     cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(LBVE_ERR_CUDA, "lbve_field_totals_noalloc: device %d beyond the %d supported",
                     dev, kMaxDevices);
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_partials);
      if (e != cudaSuccess || !p)
        return set_error(LBVE_ERR_CUDA,
                         "lbve_field_totals_noalloc: address of the static scratch on device "
                         "%d: %s",
                         dev, cudaGetErrorString(e));
      g_scratch_ptr[dev] = (double*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  int n_nodes = (int)n;
  int n_chunks = (int)((n + kChunk - 1) / kChunk);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // cudaLaunchKernel reports the error of this launch itself, so an earlier,
  // unrelated asynchronous error is neither blamed on it nor cleared
  void* args1[] = {(void*)&d_fields, (void*)&n_nodes, (void*)&scratch};
  e = cudaLaunchKernel((const void*)chunk_sums, dim3(n_chunks), dim3(kThreadsNA), args1, 0, st);
  if (e != cudaSuccess)
    return set_error(LBVE_ERR_CUDA, "lbve_field_totals_noalloc: chunk pass launch: %s",
                     cudaGetErrorString(e));
  void* args2[] = {(void*)&scratch, (void*)&n_chunks, (void*)&d_out};
  e = cudaLaunchKernel((const void*)final_sums, dim3(1), dim3(kThreadsNA), args2, 0, st);
  if (e != cudaSuccess)
    return set_error(LBVE_ERR_CUDA, "lbve_field_totals_noalloc: final pass launch: %s",
                     cudaGetErrorString(e));
  return LBVE_OK;
}

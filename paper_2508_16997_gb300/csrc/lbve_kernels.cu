// lbve_kernels.cu -- launchers of the step kernel, the deterministic float64
// reduction of per-tile partial records, and the force conversion kernel.
#include <cuda_runtime.h>

#include "lbve_internal.h"
#include "lbve_step.cuh"

namespace lbve {

template <typename R, int MODE, bool FINAL, bool MASKED, int NT>
static void launch_step_k(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                          double* d_partials, cudaStream_t st) {
  step_kernel<R, MODE, FINAL, MASKED, NT><<<n_tiles, NT, 0, st>>>(d_insts, d_tiles, parity,
                                                                  d_partials);
}

template <typename R, bool MASKED, int NT>
static int launch_step_t(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                         int mode, int flags, double* d_partials, cudaStream_t st) {
  if (n_tiles <= 0) return 0;
  const bool fin = (flags & kFinal) != 0;
  if (mode == kModeStep) {
    if (fin)
      launch_step_k<R, kModeStep, true, MASKED, NT>(d_insts, d_tiles, n_tiles, parity, d_partials,
                                                    st);
    else
      launch_step_k<R, kModeStep, false, MASKED, NT>(d_insts, d_tiles, n_tiles, parity,
                                                     d_partials, st);
  } else {
    launch_step_k<R, kModeInit, true, MASKED, NT>(d_insts, d_tiles, n_tiles, parity, d_partials,
                                                  st);
  }
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

template <typename R, int NT>
static int launch_step_m(const InstDev* d_insts, const TileDev* d_tiles, int n_tiles, int parity,
                         int mode, int flags, double* d_partials, cudaStream_t st, int masked) {
  return masked ? launch_step_t<R, true, NT>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                             d_partials, st)
                : launch_step_t<R, false, NT>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                              d_partials, st);
}

// Only the CTA sizes the host plans are instantiated; any other is refused.
int launch_step(int prec, int threads, const InstDev* d_insts, const TileDev* d_tiles,
                int n_tiles, int parity, int mode, int flags, double* d_partials, void* stream,
                int masked) {
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == 0 && threads == kThreads64)
    return launch_step_m<double, kThreads64>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                             d_partials, st, masked);
  if (prec == 0 && threads == kThreads64Tiny) {
    // tiles of at most 32 nodes: the time steps of plain tiles spread each
    // node over four warps (one lattice each), the rest runs one warp a tile
    if (!masked && mode == kModeStep && n_tiles > 0) {
      if (flags & kFinal)
        step_kernel_split<true><<<n_tiles, kSplitThreads, 0, st>>>(d_insts, d_tiles, parity,
                                                                   d_partials);
      else
        step_kernel_split<false><<<n_tiles, kSplitThreads, 0, st>>>(d_insts, d_tiles, parity,
                                                                    d_partials);
      return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
    }
    return launch_step_m<double, kThreads64Tiny>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                 d_partials, st, masked);
  }
  if (prec == 0 && threads == kThreads64Small)
    return launch_step_m<double, kThreads64Small>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                  d_partials, st, masked);
  if (prec == 1 && threads == kThreads)
    return launch_step_m<float, kThreads>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                          d_partials, st, masked);
  return -1;
}

// One CTA per instance: sum (max for the residual) the partial records of the
// instance's tiles, and the wall-pass records of its mask walls, in a fixed
// order, so totals are bit-reproducible.
__global__ void __launch_bounds__(256) reduce_kernel(const InstDev* __restrict__ insts,
                                                     int first_inst,
                                                     const double* __restrict__ partials,
                                                     double* __restrict__ totals,
                                                     int32_t* __restrict__ flags) {
  __shared__ double s[256];
  const int inst = first_inst + blockIdx.x;
  const InstDev& D = insts[inst];
  for (int j = 0; j < kDrag + 2; ++j) {
    double v = 0.0;
    if (j < kDrag)
      for (int q = D.slot_begin + threadIdx.x; q < D.slot_end; q += blockDim.x) {
        const double p = partials[(size_t)q * kPartial + j];
        v = (j == kResid) ? fmax(v, p) : v + p;
      }
    // wall record layout: drag x, drag y, in x3, out x3
    const int r = (j >= kDrag) ? j - kDrag : (j >= kWallIn && j < kResid) ? 2 + (j - kWallIn) : -1;
    if (r >= 0)
      for (int q = threadIdx.x; q < D.wall_cap; q += blockDim.x) v += D.wall_rec[(size_t)q * kWallRec + r];
    s[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        s[threadIdx.x] = (j == kResid) ? fmax(s[threadIdx.x], s[threadIdx.x + w])
                                       : s[threadIdx.x] + s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      totals[(size_t)inst * kTotals + j] = s[0];
      if (j == kNonFinite && s[0] > 0.0) flags[inst] |= 1;
    }
    __syncthreads();
  }
}

int launch_reduce(const InstDev* d_insts, int first_inst, int n_insts, const double* d_partials,
                  double* d_totals, int32_t* d_flags, void* stream) {
  if (n_insts <= 0) return 0;
  reduce_kernel<<<n_insts, 256, 0, (cudaStream_t)stream>>>(d_insts, first_inst, d_partials,
                                                           d_totals, d_flags);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

template <typename R>
__global__ void convert_force_kernel(const double* __restrict__ src, R* __restrict__ dst, int n,
                                     int stride) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dst[i] = (R)src[i];
    dst[stride + i] = (R)src[stride + i];
  }
}

int launch_convert_force(int prec, const double* d_src, void* d_dst, int n, int stride,
                         void* stream) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (blocks <= 0) return 0;
  if (prec == 0)
    convert_force_kernel<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_src, (double*)d_dst,
                                                                          n, stride);
  else
    convert_force_kernel<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_src, (float*)d_dst, n,
                                                                         stride);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

}  // namespace lbve

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
  if (prec == 2 && threads == kThreads && !masked)  // float32 pairs: plain tiles only
    return launch_step_t<df32, false, kThreads>(d_insts, d_tiles, n_tiles, parity, mode, flags,
                                                d_partials, st);
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

// Default initial fields (rho = 1, u = 0, A = I) into the float64 staging
// planes [6][stride], so that no host array is built and copied for them.
__global__ void fill_default_fields_kernel(double* __restrict__ stage, int n, int stride) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    stage[i] = 1.0;
    stage[(size_t)stride + i] = 0.0;
    stage[2 * (size_t)stride + i] = 0.0;
    stage[3 * (size_t)stride + i] = 1.0;
    stage[4 * (size_t)stride + i] = 0.0;
    stage[5 * (size_t)stride + i] = 1.0;
  }
}

int launch_fill_default_fields(double* d_stage, int n, int stride, void* stream) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (blocks <= 0) return 0;
  fill_default_fields_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_stage, n, stride);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

// Checks of the staged inputs of lbve_set_geometry, by integer tests of the
// float64 bit patterns: every force component and initial field finite (the
// exponent field is not all ones), every initial density in (0, +inf).  Sets
// bit `bit` of *flag when one fails.
__global__ void check_inputs_kernel(const double* __restrict__ force, const double* __restrict__ init,
                                    int n, int stride, int32_t* __restrict__ flag, int bit) {
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (force)
      for (int c = 0; c < 2; ++c) {
        const unsigned long long b = __double_as_longlong(force[(size_t)c * stride + i]);
        bad |= ((b >> 52) & 0x7ffull) == 0x7ffull;
      }
    if (init) {
      for (int c = 0; c < 6; ++c) {
        const unsigned long long b = __double_as_longlong(init[(size_t)c * stride + i]);
        bad |= ((b >> 52) & 0x7ffull) == 0x7ffull;
      }
      const long long r = __double_as_longlong(init[i]);
      bad |= !(r > 0 && r < 0x7ff0000000000000ll);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1 << bit);
}

int launch_check_inputs(const double* d_force, const double* d_init, int n, int stride,
                        int32_t* d_flag, int bit, void* stream) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (blocks <= 0 || (!d_force && !d_init)) return 0;
  check_inputs_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_force, d_init, n, stride, d_flag,
                                                               bit);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

template <typename R>
__global__ void convert_force_kernel(const double* __restrict__ src, R* __restrict__ dst, int n,
                                     int stride) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dst[i] = R(src[i]);
    dst[stride + i] = R(src[stride + i]);
  }
}

int launch_convert_force(int prec, const double* d_src, void* d_dst, int n, int stride,
                         void* stream) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (blocks <= 0) return 0;
  if (prec == 0)
    convert_force_kernel<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_src, (double*)d_dst,
                                                                          n, stride);
  else if (prec == 2)
    convert_force_kernel<df32><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_src, (df32*)d_dst, n,
                                                                        stride);
  else
    convert_force_kernel<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(d_src, (float*)d_dst, n,
                                                                         stride);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;  // the caller reads and clears it
}

}  // namespace lbve
